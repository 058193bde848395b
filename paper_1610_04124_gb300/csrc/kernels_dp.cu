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
// barrier per row), one CTA per column, rows cut into blocks of 32:
//   - the chain warp finalises the rows in order, lane l owning row 32 j + l of
//     block j.  At step i (start b = 32 j + i) every lane applies start b to its
//     row of block j and to its row of block j + 1 (a second running minimum,
//     so the starts of block j reach block j + 1 while block j is solved);
//     row b is then complete and its value is broadcast from lane i.  Lane 0
//     records the row's raw results in a small buffer, and at the end of the
//     block all lanes pack them into back-pointers and start contexts.  The
//     data terms of the cells (with the input-only gravity / diving penalties
//     already added) were gathered into shared memory ahead of the chain (a
//     ring of three blocks, two in the three-CTA batch shape), so the
//     sequential chain never waits on global memory.  The chain is bound by
//     its instruction issue: the bulk warps on its scheduler take no tiles.
//   - the other warps (bulk) apply the starts of every finalised block t to the
//     end rows of blocks t+2, t+3, ... (independent 32 x 32 tiles).  End-row
//     block c receives c - 1 tiles; they are split by start block between two
//     or three partial minima, the (block, partial) pairs are dealt to the
//     bulk warps largest first in snake order, and a pair always stays with
//     its warp; the chain merges the partials by (cost, start) when it
//     reaches the block.  Each bulk warp runs its pending work earliest
//     deadline first: the tile of the lowest end-row block (the chain needs it
//     soonest) or its share of the chain's data for a block, whichever the
//     chain reaches first.
//   - exact branch and bound (per-frame launches with two columns per SM):
//     a tile whose candidates are all provably dearer than a cost some
//     candidate of its end rows already reaches is skipped.  That needs the
//     newest starts first, so there a block's tiles wait until block c - 4 is
//     final and then go newest first; elsewhere they go in start order as
//     their start blocks become final.
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
#include <algorithm>
#include <climits>

#include "internal.h"
#include "real_cost.cuh"

namespace stx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBlocks = (STIXELS_MAX_HEIGHT + 31) / 32;
constexpr int kRingMax = 3;           // chain data buffers (blocks gathered ahead): 2 or 3
constexpr int kMaxSlots = 3;          // partial running minima per end row (start blocks t mod slots): 2 or 3
constexpr int kSpinLimit = 1 << 22;   // polls before a wait gives up (well over 0.1 s)

// What the bulk tiles need of one start row b, shared by every end row k >= b
// (cost terms include the previous class's code in their low bits):
//   o0 = min(V_o[b-1] + T(obj|obj), V_s[b-1] + T(obj|sky)),  o1 = the same with
//        the ordering penalty on the object term (applies iff f > ford),
//   g0 / gg / gd = V_g[b-1] + T(obj|ground) plus no penalty / the gravity
//        penalty (iff f > fhi) / the diving penalty (iff f < flo),
// so that a candidate is d + min(f > ford ? o1 : o0, f > fhi ? gg : f < flo ? gd : g0).
// (fhi >= flo - 1 holds for non-negative tolerances, so the two ground tests
// never both hold.)
struct __align__(16) BulkCtx {
    int32_t o0, o1, g0, gg, gd, ford, fhi, flo;
};

// Input-only data of row v, in two arrays: pd8[v] = PD[v] + 8 v (so that
// S + 8 n of a stixel [b, k] is pd8[k + 1] - pd8[b]) and thr[v], the gravity /
// diving thresholds at row v (penalty iff f > fhi, iff f < flo) as two int16
// halves (fhi low, flo high), clamped to [-1, 256] where that keeps every
// comparison with f in [0, 255] unchanged.
__device__ __forceinline__ int thr_hi(int32_t w) { return (int32_t)(int16_t)(w & 0xffff); }
__device__ __forceinline__ int thr_lo(int32_t w) { return w >> 16; }

// Chain data of one block j (rows B = 32 j ..): for start i and end lane l,
// {d, e_g} = the object data cost and the same plus the ground-below
// penalties, and f = the rounded mean, of the cells (B + i, B + l), i <= l
// (tri, packed by start: slot tri_slot(i) + l - i) and (B + i, B + 32 + l)
// (nxt, slot 32 i + l).  Cells past the column's end hold zeros.  One more
// start's worth of slots (tri_slot(32) = 528, nxt 1024 + l) is never written:
// the chain's look-ahead load after a block's last step reads there, so it
// needs no clamp, and never uses what it read.
struct ChainBuf {
    int2 tri[528 + 1];
    int2 nxt[1024 + 32];
    uint8_t ftri[528 + 1];
    uint8_t fnxt[1024 + 32];
};
// first triangle slot of start i: the starts before it own 32, 31, ... slots
__device__ __forceinline__ int tri_slot(int i) { return (i * (65 - i)) >> 1; }

struct SyncState {
    // bar_final[j] completes (phase 0) when the chain warp has finalised block
    // j.  A warp waiting on it is suspended in the hardware instead of
    // polling, so idle warps take no issue slots from the working ones.
    unsigned long long bar_final[kMaxBlocks];
    int32_t fin[3];              // V of the top row per class, for a bulk warp leading the tail
    int final_blocks;            // blocks the chain warp has finalised
    int abort;                   // set when a wait gave up
    int rep_state;               // cost report: 0 stixels not staged yet, 1 staged (rows may start), 2 no report
    int rep_n;                   // stixels on the path
    int rep_done;                // warps done with their rows
    long long rep_acc;           // the report's sum so far, 2^-24 units
    int qmin, qmax;              // the column's extreme Q4 codes
    int ready[kMaxBlocks];       // ready[c]: bulk tiles applied to end-row block c (of c - 1)
    int gathered[kMaxBlocks];    // gathered[j]: bulk warps done with block j's chain data
};

__device__ __forceinline__ int32_t min3(int32_t a, int32_t b, int32_t c) { return min(min(a, b), c); }

__device__ const DivTable kDivTable = make_div_table();

// Rounded mean disparity of a stixel of n rows from x = S + 8 n, clamped to
// the LUT's rows: valid Q4 input always gives f <= dmax; the clamp only keeps
// malformed caller-built LUTs (stixels_solve) inside the table.
__device__ __forceinline__ int mean_f(int32_t x, int n, const uint2* s_div, int dmax)
{
    const uint2 dm = s_div[n];
    return (int)min(__umulhi((uint32_t)x, dm.x) >> dm.y, (uint32_t)dmax);
}

// The bulk context of a start from its three previous-class terms (bo, bg, bs,
// each V_p[b-1] + T(obj|p) + code(p)), its ordering threshold and the start
// row's gravity / diving thresholds.
__device__ __forceinline__ BulkCtx make_bulk_ctx(int32_t bo, int32_t bg, int32_t bs, int32_t ford, int32_t thr,
                                                 const ModelDev& m)
{
    return BulkCtx{min(bo, bs), min(bo + m.pen_ord, bs), bg, bg + m.pen_grav, bg + m.pen_div, ford,
                   thr_hi(thr), thr_lo(thr)};
}

// Minimum of N candidates (cost, start << 8 | f) listed in ascending start
// order, ties to the earlier start, by a pairwise tree.  Result in v[0], bf[0].
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

// Warp-wide bounded wait until *p >= target (lane 0 polls, sleeping between
// polls with a back-off up to max_ns, at most `limit` polls).  Returns false
// if the wait gave up or another warp did; the caller then stops.
__device__ __forceinline__ bool wait_geq(volatile int* p, int target, volatile int* abort_flag, int max_ns,
                                         int limit = kSpinLimit)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        int it = 0, ns = 8;
        while (*p < target) {
            if (*abort_flag) { ok = 0; break; }
            if (++it > limit) { *abort_flag = 1; ok = 0; break; }
            __nanosleep(ns);
            ns = min(2 * ns, max_ns);
        }
    }
    ok = __shfl_sync(kFull, ok, 0);
    __threadfence_block();
    return ok != 0;
}

// Shared-memory barriers (PTX mbarrier), each used for one phase per column.
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(unsigned long long* b, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_inval(unsigned long long* b)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

// arrive (release: this thread's earlier writes are visible to the waiters)
__device__ __forceinline__ void bar_arrive(unsigned long long* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}

// Whether phase 0 of the barrier has completed (acquire); the thread may be
// suspended for up to the hint (ns) while it has not.
__device__ __forceinline__ bool bar_try_wait(unsigned long long* b, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(hint_ns)
                 : "memory");
    return ok != 0;
}

// Warp-wide bounded wait for phase 0 of a barrier (lane 0 waits, suspended
// between tries, at most `limit` tries).  Returns false if the wait gave up
// or another warp did; the caller then stops.
__device__ __forceinline__ bool wait_bar(unsigned long long* b, volatile int* abort_flag, int limit = kSpinLimit)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        int it = 0;
        while (!bar_try_wait(b, 1000)) {
            if (*abort_flag) { ok = 0; break; }
            if (++it > limit) { *abort_flag = 1; ok = 0; break; }
        }
    }
    ok = __shfl_sync(kFull, ok, 0);
    __syncwarp();
    __threadfence_block();
    return ok != 0;
}

__host__ __device__ size_t dp_smem_bytes(int H, int ring, int slots)
{
    const size_t HP = (size_t)((H + 3) & ~3);
    return sizeof(BulkCtx) * HP + sizeof(int4) * HP + sizeof(int32_t) * 2 * (HP + 4) + sizeof(int2) * (HP + 4) +
           sizeof(uint2) * (HP + 4) + sizeof(int32_t) * 2 * slots * HP + sizeof(ChainBuf) * ring +
           sizeof(SyncState);
}

// The SyncState of a CTA's shared memory laid out as dp_column lays it out
// (it is the last member)
__device__ __forceinline__ SyncState* dp_sync_state(int32_t* sm, int H, int ring, int slots)
{
    return reinterpret_cast<SyncState*>(reinterpret_cast<char*>(sm) + dp_smem_bytes(H, ring, slots) - sizeof(SyncState));
}

// Gathers the chain data of the block starting at row B into cb.  Warp w of
// nw takes the starts b = B + i for i = w, w + nw, ...; lane l computes the
// cells (b, B + l) (triangle slot i 32 + l, written only for i <= l) and
// (b, B + 32 + l) (next-block slot), two starts' loads in flight at a time.
// Every lane runs the same instructions: an invalid cell (end row above the
// column or below the start) is evaluated at a clamped end row, so that its
// loads stay inside the column, and stored as zeros (cells below the start
// are not stored).  Starts past the block or the column are skipped (the
// chain never reads them).
__device__ __forceinline__ void gather_chain(ChainBuf* cb, int B, int H, int P, const int32_t* __restrict__ po_col,
                                             const int32_t* s_pd8, const int32_t* s_thr, const uint2* s_div,
                                             int dmax, int32_t pen_grav, int32_t pen_div, int w, int nw, int lane)
{
    const int k0 = B + lane, k1 = B + 32 + lane;
    const bool in0 = k0 < H, in1 = k1 < H;
    const int kh0 = min(k0, H - 1), kh1 = min(k1, H - 1);
    const int32_t x0 = s_pd8[kh0 + 1], x1 = s_pd8[kh1 + 1];
#pragma unroll 1
    for (int i0 = w; i0 < 32; i0 += 2 * nw) {
        int32_t lo[4], hi[4];
        int fv[4];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            // a start past the block or the column repeats a valid one (not stored)
            const int b = min(B + min(i0 + r * nw, 31), H - 1);
            const int32_t pb = s_pd8[b];
            const int f0 = mean_f(x0 - pb, max(kh0 - b + 1, 1), s_div, dmax);
            const int f1 = mean_f(x1 - pb, kh1 - b + 1, s_div, dmax);     // kh1 >= b always
            const int32_t* row0 = po_col + f0 * P;
            const int32_t* row1 = po_col + f1 * P;
            lo[2 * r] = __ldg(row0 + b);
            hi[2 * r] = __ldg(row0 + kh0 + 1);
            lo[2 * r + 1] = __ldg(row1 + b);
            hi[2 * r + 1] = __ldg(row1 + kh1 + 1);
            fv[2 * r] = f0;
            fv[2 * r + 1] = f1;
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = i0 + r * nw, b = B + i;
            if (i < 32 && b < H) {                                       // uniform across the warp
                const int32_t thr = s_thr[b];
                const int fhi = thr_hi(thr), flo = thr_lo(thr);
                const bool ok0 = i <= lane && in0;
                const int f0 = ok0 ? fv[2 * r] : 0, f1 = in1 ? fv[2 * r + 1] : 0;
                const int32_t d0 = ok0 ? hi[2 * r] - lo[2 * r] : 0;
                const int32_t d1 = in1 ? hi[2 * r + 1] - lo[2 * r + 1] : 0;
                const int32_t g0 = ok0 ? (f0 > fhi ? pen_grav : 0) + (f0 < flo ? pen_div : 0) : 0;
                const int32_t g1 = in1 ? (f1 > fhi ? pen_grav : 0) + (f1 < flo ? pen_div : 0) : 0;
                if (i <= lane) {
                    const int e = tri_slot(i) + lane - i;
                    cb->tri[e] = make_int2(d0, d0 + g0);
                    cb->ftri[e] = (uint8_t)f0;
                }
                cb->nxt[i * 32 + lane] = make_int2(d1, d1 + g1);
                cb->fnxt[i * 32 + lane] = (uint8_t)f1;
            }
        }
    }
}

constexpr int kReportWarps = 4;       // bulk warps that share the cost report's rows

// The end of a column, by one warp once the chain has finalised the last
// block (the chain warp itself, or bulk warp 0): it takes the top row's best
// class (ties object < ground < sky), backtracks from it through the
// back-pointers (Sec. 3.3, Sec. 5.4), writes the stixel list bottom -> top
// and the output records, then the stixel part of the cost report (priors
// and each stixel's pixel-cost constants, staged for the rows).  vo, vg, vs:
// V of the top row per class.  `a` is the CTA's shared-memory copy of the
// arguments (the tail reads many of them, once each).  A column with no
// feasible segmentation is recorded in the error word with an empty column.
__device__ __forceinline__ void lead_column_end(const DpArgs& a, int col, int H, SyncState* sync, const int4* s_bp,
                                                const int32_t* s_pd8, const int32_t* s_thr, const uint2* s_div,
                                                int32_t* s_seg, int lane, int32_t vo, int32_t vg, int32_t vs)
{
    int c = 0;
    int32_t best = vo;
    if (vg < best) { best = vg; c = 1; }
    if (vs < best) { best = vs; c = 2; }
    if (best >= kBig) {
        if (lane == 0) {
            a.counts[col] = 0;
            if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
            if (a.cost_fixed) a.cost_fixed[col] = kBig;
            atomicOr(a.err, STIXELS_ERR_INFEASIBLE);
            __threadfence_block();
            *(volatile int*)&sync->rep_state = 2;
        }
        return;
    }
    // one walk from the top row (lane 0), the stixels top -> bottom into
    // s_seg[H..2H); the lanes then put them bottom -> top into s_seg[0..n)
    // and write the output records
    int32_t* top_down = s_seg + H;
    int n = 0;
    if (lane == 0) {
        const int32_t* bp_all = reinterpret_cast<const int32_t*>(s_bp);
        for (int k = H - 1, cc = c; k >= 0 && cc < 3 && n < H;) {
            const int32_t bp = bp_all[4 * k + cc];
            const int b = min(bp >> 2, k);               // b <= k for a solved column; keeps the walk finite
            top_down[n++] = (b << 13) | (k << 2) | cc;
            k = b - 1;
            cc = bp & 3;
        }
        a.counts[col] = n;
        if (n > a.cap) atomicOr(a.err, STIXELS_ERR_CAPACITY);
        if (a.cost_fixed) a.cost_fixed[col] = best;
    }
    n = __shfl_sync(kFull, n, 0);
    __syncwarp();
    stixel_t* out = a.stixels + (size_t)col * a.cap;
    for (int i = lane; i < n; i += 32) {
        const int w = top_down[n - 1 - i];
        s_seg[i] = w;
        if (i < a.cap) {
            const int b = w >> 13, k = (w >> 2) & 2047;
            const int nrows = k - b + 1;
            const int32_t S = s_pd8[k + 1] - s_pd8[b] - 8 * nrows;
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
    __syncwarp();
    if (!a.cost) return;
    const float* __restrict__ k_obj = real_k_obj(a.rows.real_model);
    const float* __restrict__ inv_obj = k_obj + a.F;
    auto kinv = [&](int f, bool valid) {
        return valid ? make_float2(__ldg(k_obj + f), __ldg(inv_obj + f)) : make_float2(0.f, 0.f);
    };
    auto thr = [&](int b) {
        const int32_t t = s_thr[b];
        return make_int2((int32_t)(int16_t)(t & 0xffff), t >> 16);
    };
    const long long pri = warp_sum64(report_stixels(s_seg, n, s_pd8, s_div, a, H, lane, kinv, thr));
    if (lane == 0) {
        sync->rep_acc = pri;
        sync->rep_n = n;
        __threadfence_block();
        *(volatile int*)&sync->rep_state = 1;
    }
}

// The rows of the cost report (Eq. 4 per pixel under the staged stixels), by
// kReportWarps bulk warps: role r takes the blocks of 32 rows r, r +
// kReportWarps, ...; the sums go into one exact integer and the last warp to
// finish writes the column's cost.  The warps first wait (suspended) for the
// chain's last block, then briefly poll for the staged stixels.
__device__ __forceinline__ void report_column_rows(const DpArgs& a, int col, int H, SyncState* sync,
                                                   const int32_t* s_pd8, const int32_t* s_seg, int lane, int role)
{
    if (!a.cost) return;
    const int NB = (H + 31) >> 5;
    // this warp's first rows' tables are loaded before the waits
    RowTables pre;
    load_rows(pre, a.rows.fg, H, lane, role, kReportWarps);
    if (!wait_bar(&sync->bar_final[NB - 1], &sync->abort)) return;     // the chain reports the failure
    if (!wait_geq(&sync->rep_state, 1, &sync->abort, 16)) {
        if (lane == 0) {
            a.cost[col] = __int_as_float(0x7f800000);
            atomicOr(a.err, STIXELS_ERR_TIMEOUT);
        }
        return;
    }
    if (*(volatile int*)&sync->rep_state != 1) return;
    const int n = *(volatile int*)&sync->rep_n;
    const long long sum = warp_sum64(report_rows(s_seg, n, s_pd8, a, H, lane, role, kReportWarps, &pre));
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&sync->rep_acc), (unsigned long long)sum);
        __threadfence_block();
        if (atomicAdd(&sync->rep_done, 1) == kReportWarps - 1) {
            const long long total = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&sync->rep_acc), 0ull);
            a.cost[col] = __ll2float_rn(total) * (1.0f / kReportUnits);
        }
    }
}

// The same as calls (the persistent kernel's shape: measured faster there
// than inlined, and with a bulk warp leading the tail)
__device__ __noinline__ void lead_column_end_call(const DpArgs& a, int col, int H, SyncState* sync, const int4* s_bp,
                                                  const int32_t* s_pd8, const int32_t* s_thr, const uint2* s_div,
                                                  int32_t* s_seg, int lane, int32_t vo, int32_t vg, int32_t vs)
{
    lead_column_end(a, col, H, sync, s_bp, s_pd8, s_thr, s_div, s_seg, lane, vo, vg, vs);
}

__device__ __noinline__ void report_column_rows_call(const DpArgs& a, int col, int H, SyncState* sync,
                                                     const int32_t* s_pd8, const int32_t* s_seg, int lane, int role)
{
    report_column_rows(a, col, H, sync, s_pd8, s_seg, lane, role);
}

// Solves column `col` of frame `a` with all NW warps of the CTA (one chain
// warp, NW - 1 bulk warps); `sm` is the CTA's dynamic shared memory
// (dp_smem_bytes with the same ring, 2 or 3 chain buffers, and slots, 2 or 3
// partial minima per end row).  Every warp
// returns from here; the caller synchronises before reusing `sm`.
// kChainTail: the chain warp leads the column's tail as soon as it has
// finalised the last block (the per-frame kernel; measured 94.2 -> 90.1 us at
// 1024x440), else bulk warp 0 does, through calls (the persistent kernel,
// where the chain-led tail measured 10 % slower: 13.2 K against 11.9 K frames/s
// for 32 1024x440 frames, and the bulk-led one 13.9 K).
template <int NW, bool kStdTrans, bool kChainTail>
__device__ __forceinline__ void dp_column(const DpArgs& a, const DpArgs& ta, const int col, const int ring,
                                          const int slots, const int window, int32_t* sm, const int chain)
{
    constexpr int kWarps = NW;
    constexpr int kThreads = NW * 32;
    constexpr int kBulk = NW - 1;                   // warps besides the chain warp
    // the tile dealing below leaves out the bulk warps on the chain warp's
    // scheduler (warp index congruent mod 4): NW / 4 - 1 of them
    static_assert(NW % 4 == 0 && NW >= 8, "whole schedulers of warps");
    static_assert(kReportWarps == 4 && NW - 1 > 4, "the report's warps are bulk warps 0, 1, 2, 4");
    constexpr int kTile = kBulk - (NW / 4 - 1);    // bulk warps that take tiles
    constexpr bool kQuietExit = NW >= 16;
    constexpr int kGather = kQuietExit ? kTile : kBulk;   // warps that share each gather
    const int H = a.H, P = a.P, F = a.F;
    const int HP = (H + 3) & ~3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ModelDev& m = a.m;
    // `chain` is the chain warp (0 .. 3); the other warps are bulk warps
    // 0 .. kBulk-1.  The per-frame kernel puts it on warp 0 in every CTA (two
    // CTAs sharing an SM then have both chains on one scheduler, next to warps
    // that take no tiles: 90.0 vs 91.2 us at two columns per SM); the batch
    // kernel, up to three CTAs per SM, rotates it with the column.
    const int bulk_id = (warp - chain - 1 + kWarps) % kWarps;

    BulkCtx* s_ctx = reinterpret_cast<BulkCtx*>(sm);                   // [HP]
    int4* s_bp = reinterpret_cast<int4*>(s_ctx + HP);                  // [HP] back-pointers b << 2 | p per class
    int32_t* s_pd8 = reinterpret_cast<int32_t*>(s_bp + HP);            // [HP + 4], v = 0..H
    int32_t* s_thr = s_pd8 + HP + 4;                                   // [HP + 4]
    int2* s_gs = reinterpret_cast<int2*>(s_thr + HP + 4);              // [HP + 4] {PG[v], PS[v]}, v = 0..H
    uint2* s_div = reinterpret_cast<uint2*>(s_gs + HP + 4);            // [HP + 4], index n = 1..H
    // [slots][HP] object running minima over the start blocks t = s (mod slots)
    int32_t* s_runv = reinterpret_cast<int32_t*>(s_div + HP + 4);
    int32_t* s_runbf = s_runv + slots * HP;                            // [slots][HP] start << 8 | f
    ChainBuf* s_cb = reinterpret_cast<ChainBuf*>(s_runbf + slots * HP);    // [ring]
    SyncState* sync = reinterpret_cast<SyncState*>(s_cb + ring);
    volatile int* v_final = &sync->final_blocks;
    volatile int* v_abort = &sync->abort;
    const int NB = (H + 31) >> 5;

    const int32_t* po_col = a.po + (size_t)col * F * P;
    const int32_t* pg_col = a.pg + (size_t)col * P;
    const int32_t* ps_col = a.ps + (size_t)col * P;
    const int32_t* thr_row = rows_thr(a.rows.fg, H);   // gravity / diving thresholds of each row
    for (int n = 1 + threadIdx.x; n <= H; n += kThreads) {
        const DivMagic dm = kDivTable.v[n];
        s_div[n] = make_uint2(dm.m, dm.s);
    }
    {
        // what the column's cost report reads at the end (the row tables and
        // the unrounded model) is fetched into L2 now, while the DP runs
        const char* rb = reinterpret_cast<const char*>(a.rows.fg);
        const int nr = (int)rows_arrays_bytes(H);
        for (int o = 128 * threadIdx.x; o < nr; o += 128 * kThreads) asm volatile("prefetch.global.L2 [%0];" ::"l"(rb + o));
        const char* mb = reinterpret_cast<const char*>(real_k_obj(a.rows.real_model));
        const int nm = 8 * F;
        for (int o = 128 * threadIdx.x; o < nm; o += 128 * kThreads) asm volatile("prefetch.global.L2 [%0];" ::"l"(mb + o));
    }
    // the tables: from here on this kernel reads what the LUT kernel wrote
    grid_dependency_wait();
    for (int v = threadIdx.x; v <= H; v += kThreads) {
        int32_t thr = 0;
        if (v < H) {
            thr = thr_row[v];
#pragma unroll
            for (int q = 0; q < slots; ++q) {
                s_runv[q * HP + v] = INT_MAX;
                s_runbf[q * HP + v] = 0;
            }
        }
        s_gs[v] = make_int2(pg_col[v], ps_col[v]);
        s_pd8[v] = a.pd[(size_t)col * P + v] + 8 * v;
        s_thr[v] = thr;
    }
    if (threadIdx.x < kMaxBlocks) {
        sync->ready[threadIdx.x] = 0;
        sync->gathered[threadIdx.x] = 0;
        bar_init(&sync->bar_final[threadIdx.x], 1);
    }
    if (threadIdx.x == 0) {
        sync->final_blocks = 0;
        sync->abort = 0;
        sync->rep_state = 0;
        sync->rep_done = 0;
        sync->rep_acc = 0;
        sync->qmin = INT_MAX;
        sync->qmax = INT_MIN;
        // start 0 carries the first-stixel prior (code 3 = no previous stixel)
        s_ctx[0] = make_bulk_ctx(m.first[0] + kNoneCode, kBig, kBig, INT_MAX, s_thr[0], m);
    }
    __syncthreads();
    if (window < kMaxBlocks) {
        // (tiles pruned by the bound) the column's code range: every
        // stixel's rounded mean lies between round(min q / 16) and
        // round(max q / 16), the object rows the tile bound takes its minimum
        // over (the LUT kernel writes no others)
        int lo = INT_MAX, hi = INT_MIN;
        for (int v = threadIdx.x; v < H; v += kThreads) {
            const int qv = s_pd8[v + 1] - s_pd8[v] - 8;
            lo = min(lo, qv);
            hi = max(hi, qv);
        }
        lo = __reduce_min_sync(kFull, lo);
        hi = __reduce_max_sync(kFull, hi);
        if (lane == 0) {
            atomicMin(&sync->qmin, lo);
            atomicMax(&sync->qmax, hi);
        }
        __syncthreads();
    }

    // Apply the 32 starts of finalised block t to end-row block jc (a bulk tile):
    // lane l owns end row k = 32 jc + l; the starts go in four groups of 8
    // (16 gathers in flight), each merged by a pairwise tree, then folded into
    // the running minimum in start order.  The group loop stays rolled to keep
    // the kernel's code small.
    auto bulk_tile = [&](int t, int jc, bool older) {
        const int k = 32 * jc + lane;
        const bool kv = k < H;
        const int kk = kv ? k : H - 1;
        int32_t* runv = s_runv + (t % slots) * HP;
        int32_t* runbfv = s_runbf + (t % slots) * HP;
        int32_t run = INT_MAX, runbf = 0;
        if (kv) { run = runv[k]; runbf = runbfv[k]; }
        const int32_t x1 = s_pd8[kk + 1];
        const int32_t* hi_base = po_col + kk + 1;           // PO[f][k + 1] = hi_base[f P]
        // older: the tile's starts come before (below) every start already in
        // this partial minimum, so groups go in descending order and "<="
        // lets the earlier start win on equal cost; otherwise they come after
        // every one of them, in ascending order with "<"
#pragma unroll 1
        for (int gi = 0; gi < 4; ++gi) {
            const int g = older ? 3 - gi : gi;
            const int b0 = 32 * t + 8 * g;
            const uint2* divp = s_div + (kk + 1 - b0);      // s_div[k + 1 - b] = divp[-i], b = b0 + i
            const int32_t* lo_base = po_col + b0;           // PO[f][b] = lo_base[f P + i]
            const int4 pa = *reinterpret_cast<const int4*>(s_pd8 + b0);
            const int4 pb = *reinterpret_cast<const int4*>(s_pd8 + b0 + 4);
            const int32_t pdv[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
            int32_t lo[8], hi[8], fv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint2 dm = divp[-i];
                const int f = (int)min(__umulhi((uint32_t)(x1 - pdv[i]), dm.x) >> dm.y, (uint32_t)m.dmax);
                lo[i] = __ldg(lo_base + (size_t)f * P + i);
                hi[i] = __ldg(hi_base + (size_t)f * P);
                fv[i] = f;
            }
            int32_t cv[8], cbf[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int b = b0 + i;
                const BulkCtx c = s_ctx[b];
                const int f = fv[i];
                const int32_t o = f > c.ford ? c.o1 : c.o0;
                const int32_t gr = f > c.fhi ? c.gg : (f < c.flo ? c.gd : c.g0);
                cv[i] = min(o, gr) + (hi[i] - lo[i]);
                cbf[i] = (b << 8) | f;
            }
            tree_min<8>(cv, cbf);
            if (cv[0] < run || (older && cv[0] == run)) { run = cv[0]; runbf = cbf[0]; }
        }
        if (kv) { runv[k] = run; runbfv[k] = runbf; }
    };

    // Whether no candidate of tile (t, jc) can be the best object stixel of
    // any of the block's end rows (exact branch and bound): every stixel of
    // the tile spans the rows cs = 32 t + 31 .. 32 jc, so its cost is at least
    // the best context of its start, plus the cheapest of those core rows'
    // data over all f (a difference of two LUT rows), plus the per-pixel floor
    // of the model for its other rows.  The tile is skipped when that bound
    // exceeds, on every end row, a cost some candidate already reaches (any
    // partial minimum; tiles come newest start first, so these are low early).
    auto tile_bounded = [&](int t, int jc) -> bool {
        const int k = 32 * jc + lane;
        const int b = 32 * t + lane;
        const BulkCtx cx = s_ctx[b];
        int32_t lb = min(min(min(cx.o0, cx.o1), min(cx.g0, cx.gg)), cx.gd) - b * a.pixel_floor;
        lb = __reduce_min_sync(kFull, lb);
        const int cs = 32 * t + 31;
        // the core difference of every f a stixel of the column can have,
        // lane l taking f = f_lo + l + 32 j (clamped to f_hi, which repeats
        // the last one): all loads in flight at once
        // (malformed codes from a caller's tables: the whole range)
        const int qlo = sync->qmin, qhi = sync->qmax;
        const int f_lo = qlo < 0 ? 0 : min((qlo + 8) >> 4, F - 1);
        const int f_span = (qlo < 0 ? F - 1 : min((qhi + 8) >> 4, F - 1)) - f_lo;
        int32_t cm = INT_MAX;
        const int32_t* core_hi = po_col + 32 * jc + 1;
        const int32_t* core_lo = po_col + cs;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const size_t o = (size_t)(f_lo + min(lane + 32 * j, f_span)) * P;
            cm = min(cm, __ldg(core_hi + o) - __ldg(core_lo + o));
        }
        cm = __reduce_min_sync(kFull, cm);
        bool beat = true;
        if (k < H) {
            const int32_t bound = lb + cs * a.pixel_floor + cm + (k - 32 * jc) * a.pixel_floor;
            int32_t rv = s_runv[k];
#pragma unroll
            for (int q = 1; q < slots; ++q) rv = min(rv, s_runv[q * HP + k]);
            beat = bound > rv;
        }
        return __all_sync(kFull, beat);
    };

    if (warp != chain) {
        // ---------------------------------------------------------------- bulk warps
        // End-row block c receives c - 1 tiles, split by start block into
        // `slots` partial minima (t = s mod slots) so that two or three warps share a
        // block's sequence of tiles.  The (block, slot) items are dealt, largest
        // block first, to the tile warps in snake order (rounds of kTile items,
        // alternating direction), which keeps the per-warp work balanced; lane l
        // of a tile warp holds its round-l item and the next start block due.
        // The bulk warps that share the chain warp's scheduler (warp index
        // congruent to the chain's mod 4: bulk ids 3, 7, 11) take no tiles, only
        // their share of the gathers, so the chain's dependent steps are not
        // starved of issue slots there.
        static_assert(32 * kTile >= kMaxSlots * (kMaxBlocks - 2), "every (block, slot) item has a tile warp");
        const bool quiet = ((bulk_id + 1) & 3) == 0;
        const int tile_id = bulk_id - ((bulk_id + 1) >> 2);
        // In the one-column-per-SM shape the quiet warps leave at once and the
        // tile warps also do the gathers (measured: a lone column 67.6 -> 63.5
        // us); with two columns per SM the gathers keep all bulk warps.
        if (kQuietExit && quiet) return;
        const int snake = (lane & 1) ? kTile - 1 - tile_id : tile_id;
        const int item = lane * kTile + snake;
        const int my_c = NB - 1 - item / slots;
        const int slot = item % slots;
        // The item's tiles are its slot's start blocks t <= my_c - 2.  The
        // item opens once block my_c - 2 - window is final: its tiles up to
        // that block go newest first (so that the bound above prunes the older
        // ones with the newer ones' minima), then the `window` newer ones in
        // order as their start blocks become final.  my_t is the next tile
        // due (-1 once none is left), my_old whether it is still in the first
        // part.
        const int newest = my_c - 2;
        const int split = newest - window;                   // the last tile of the first part
        auto slot_top = [&](int t) { return t >= slot ? slot + (t - slot) / slots * slots : -1; };
        auto slot_after = [&](int t) {                       // the first tile of the slot above t
            const int u = slot + ((t + 1 - slot + slots - 1) / slots) * slots;
            return u <= newest ? u : -1;
        };
        const int my_first = slot_top(split);                // the item's first tile (newest of the first part)
        const int my_after = slot_after(max(split, -1));     // the first tile of the second part
        int my_t = my_first;
        bool my_old = my_t >= 0;
        if (!my_old) my_t = my_after;
        const bool mine = !quiet && my_c >= 2;
        // pending work, earliest deadline first: the next tile of the lowest
        // owned end-row block, once it is open (block my_c - 3 final) and its
        // start block is final, or this warp's share of the chain data of
        // block next_g (its ring slot is free once block next_g - ring is
        // final)
        int next_g = 0;
        for (;;) {
            const int vf = __shfl_sync(kFull, lane == 0 ? *v_final : 0, 0);     // final blocks
            if (*v_abort) break;
            const bool pending = mine && my_t >= 0;
            const unsigned work = __ballot_sync(kFull, pending && vf >= my_c - 1 - window && vf > my_t);
            const bool all_done = __ballot_sync(kFull, pending) == 0;
            // owned blocks decrease with the lane: the lowest block is the highest lane
            const int wl = work ? 31 - __clz(work) : -1;
            const int jc_work = wl >= 0 ? __shfl_sync(kFull, my_c, wl) : -1;
            const bool g_open = next_g < NB && vf >= next_g - ring + 1;
            if (g_open && (jc_work < 0 || next_g <= jc_work)) {
                gather_chain(s_cb + next_g % ring, 32 * next_g, H, P, po_col, s_pd8, s_thr, s_div, m.dmax,
                             m.pen_grav, m.pen_div, kQuietExit ? tile_id : bulk_id, kGather, lane);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) atomicAdd(&sync->gathered[next_g], 1);
                ++next_g;
                continue;
            }
            if (jc_work >= 0) {
                const int t = __shfl_sync(kFull, my_t, wl);
                const bool older = __shfl_sync(kFull, my_old ? 1 : 0, wl) != 0;
                // the bound pays off only against minima already found: not
                // for an item's first tile, nor for the newest ones, which
                // the older ones' minima rarely beat
                const bool check = older && t != __shfl_sync(kFull, my_first, wl);
                if (!(check && tile_bounded(t, jc_work))) bulk_tile(t, jc_work, older);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) atomicAdd(&sync->ready[jc_work], 1);
                if (lane == wl) {
                    if (my_old && t - slots >= 0) my_t = t - slots;
                    else if (my_old) { my_old = false; my_t = my_after; }
                    else my_t = t + slots <= newest ? t + slots : -1;
                }
                continue;
            }
            if (all_done && next_g >= NB) break;
            if (vf >= NB || !wait_bar(&sync->bar_final[vf], v_abort)) break;
        }
        // the rows of the cost report go to bulk warps 0, 1, 2 and 4 (none
        // shares the chain's scheduler, where the other column of the SM may
        // still be running its chain, and none leaves early)
        const int role = bulk_id < 3 ? bulk_id : (bulk_id == 4 ? 3 : -1);
        if constexpr (kChainTail) {
            if (role >= 0) report_column_rows(ta, col, H, sync, s_pd8, s_runv, lane, role);
        } else {
            if (role == 0 && wait_bar(&sync->bar_final[NB - 1], v_abort))
                lead_column_end_call(ta, col, H, sync, s_bp, s_pd8, s_thr, s_div, s_runv, lane, sync->fin[0],
                                     sync->fin[1], sync->fin[2]);
            if (role >= 0) report_column_rows_call(ta, col, H, sync, s_pd8, s_runv, lane, role);
        }
        return;
    }

    // -------------------------------------------------------------------- chain warp
    // transition priors with the previous-class codes folded in
    const int32_t T_oo = m.trans[0][0], T_og = m.trans[0][1] + 1, T_os = m.trans[0][2] + 2;
    const int32_t T_go = m.trans[1][0], T_gg = m.trans[1][1] + 1, T_gs = m.trans[1][2] + 2;
    const int32_t T_so = m.trans[2][0], T_sg = m.trans[2][1] + 1, T_ss = m.trans[2][2] + 2;
    const int ord_off = m.ord_off;                  // 16 f > 16 f' + 16 eps  <=>  f > f' + floor(eps)
    const int32_t pen_ord = m.pen_ord;
    // per-row results of the current block, written by lane 0 at each step and
    // packed into back-pointers / start contexts by all lanes at the block's end
    // (a separate array, so these stores do not hold back the next steps' loads)
    __shared__ int4 s_raw[32];                      // {object value, start << 8 | f, ground, sky}
    __shared__ int2 s_raw2[32];                     // {ground start, sky start}
    // carried state (uniform across lanes): V of the last finalised row, f of
    // its best object stixel, and the ground / sky running minima
    int32_t vo_p = 0, vg_p = 0, vs_p = 0, fo_p = 0;
    int32_t rg = INT_MAX, rgb = 0, rs = INT_MAX, rsb = 0;
    // lane l's running minimum for row 32 (j + 1) + l over the starts of block j
    int32_t run2 = INT_MAX, run2bf = 0;
    bool aborted = false;

    for (int j = 0; j < NB; ++j) {
        const int B = 32 * j;
        if (!wait_geq(&sync->gathered[j], kGather, v_abort, 16)) { aborted = true; break; }
        if (j >= 2 && !wait_geq(&sync->ready[j], j - 1, v_abort, 16)) { aborted = true; break; }
        const ChainBuf* cb = s_cb + (j % ring);
        const int nb = min(32, H - B);
        const int k = B + lane;
        // starts of blocks <= j-2 (bulk tiles), then those of block j-1 (run2):
        // ascending starts with strict "<" keep the earliest start on ties
        int32_t run = INT_MAX, runbf = 0;
        if (lane < nb) {
            // merge the partial minima by (cost and class, start): the minimum
            // over all their starts with ties to the earliest start
            run = s_runv[k];
            runbf = s_runbf[k];
#pragma unroll
            for (int q = 1; q < slots; ++q) {
                const int32_t v = s_runv[q * HP + k], bf = s_runbf[q * HP + k];
                if (v < run || (v == run && (bf >> 8) < (runbf >> 8))) { run = v; runbf = bf; }
            }
        }
        if (run2 < run) { run = run2; runbf = run2bf; }
        run2 = INT_MAX; run2bf = 0;
        // inputs of one step, loaded a step ahead so that shared-memory latency
        // overlaps the previous step (the ground / sky prefix at b comes from
        // the step before, which loaded it as its b + 1)
        struct StepIn {
            int2 gs1, de, de2;
            int ff, ff2;
        };
        // ts = tri_slot(i), carried from step to step
        auto load_in = [&](int i, int ts) {
            StepIn x;
            x.gs1 = s_gs[B + i + 1];
            // a lane below the start reads the cell (i, i): its rows are final,
            // so what it then computes is never used
            const int e = ts + max(lane - i, 0);
            x.de = cb->tri[e];
            x.ff = cb->ftri[e];
            x.de2 = cb->nxt[i * 32 + lane];
            x.ff2 = cb->fnxt[i * 32 + lane];
            return x;
        };
        // one start of the block, start row b = B + i; `first` is set only for
        // b = 0, whose candidates carry the first-stixel prior
        auto step = [&](int i, int2 gs0, const StepIn& x, bool first) {
            const int b = B + i;
            int32_t bo, bg, bs, ford, ag, as;
            if (first) {
                bo = m.first[0] + kNoneCode; bg = kBig; bs = kBig; ford = INT_MAX;
                ag = m.first[1] + kNoneCode - gs0.x;
                as = m.first[2] + kNoneCode - gs0.y;
            } else {
                bo = vo_p + T_oo; bg = vg_p + T_og; bs = vs_p + T_os; ford = fo_p + ord_off;
                if (kStdTrans) {
                    ag = vo_p + T_go - gs0.x;
                    as = min(vo_p + T_so, vg_p + T_sg) - gs0.y;
                } else {
                    ag = min3(vo_p + T_go, vg_p + T_gg, vs_p + T_gs) - gs0.x;
                    as = min3(vo_p + T_so, vg_p + T_sg, vs_p + T_ss) - gs0.y;
                }
            }
            // every lane: start b applied to its rows of blocks j and j + 1; the
            // object and sky terms add the same data cost, so
            // min(bo [+ ordering] + d, bs + d) = min(bo [+ ordering], bs) + d
            const int32_t o_lo = min(bo, bs), o_hi = min(bo + pen_ord, bs);
            const int32_t cand = min((x.ff > ford ? o_hi : o_lo) + x.de.x, bg + x.de.y);
            if (cand < run) { run = cand; runbf = (b << 8) | x.ff; }
            const int32_t cand2 = min((x.ff2 > ford ? o_hi : o_lo) + x.de2.x, bg + x.de2.y);
            if (cand2 < run2) { run2 = cand2; run2bf = (b << 8) | x.ff2; }
            if (ag < rg) { rg = ag; rgb = b; }
            if (as < rs) { rs = as; rsb = b; }
            // row b is complete (lane i has applied every start <= b)
            const int32_t r = __shfl_sync(kFull, run, i);
            const int32_t bf = __shfl_sync(kFull, runbf, i);
            const int32_t gr = x.gs1.x + rg;
            const int32_t sk = x.gs1.y + rs;
            vo_p = min(r & ~3, kBig);
            vg_p = min(gr & ~3, kBig);
            vs_p = min(sk & ~3, kBig);
            fo_p = bf & 255;
            if (lane == 0) {
                s_raw[i] = make_int4(r, bf, gr, sk);
                s_raw2[i] = make_int2(rgb, rsb);
            }
        };
        int2 gs0 = s_gs[B];
        int ts = 0;
        StepIn cur = load_in(0, 0);
        int i = 0;
        if (j == 0) {
            // start 0, with the first-stixel prior, outside the loop
            const StepIn nx = load_in(1, 32);            // 1 = nb: read, never used
            step(0, gs0, cur, true);
            gs0 = cur.gs1;
            cur = nx;
            ts = 32;
            i = 1;
        }
        // unrolled by 4 in the per-frame kernel, by 2 in the persistent one
        // (measured: a step of the chain alone 136 -> 107 cycles with start 0
        // peeled and 4 steps per iteration; 1024x440 DP 90.1 -> 88.1 us, while
        // 32 batched frames ran at 13.7 K against 13.9 K frames/s unrolled by 4)
#pragma unroll(kChainTail ? 4 : 2)
        for (; i < nb; ++i) {
            const int tsn = ts + 32 - i;                 // tri_slot(i + 1)
            const StepIn nx = load_in(i + 1, tsn);       // i + 1 = nb: read, never used
            step(i, gs0, cur, false);
            gs0 = cur.gs1;
            cur = nx;
            ts = tsn;
        }
        __syncwarp();
        // the block's back-pointers and the contexts of the starts that follow its rows
        if (lane < nb) {
            const int4 w = s_raw[lane];
            const int2 w2 = s_raw2[lane];
            s_bp[k] = make_int4(((w.y >> 8) << 2) | (w.x & 3), (w2.x << 2) | (w.z & 3), (w2.y << 2) | (w.w & 3), 0);
            if (k + 1 < H)
                s_ctx[k + 1] = make_bulk_ctx(min(w.x & ~3, kBig) + T_oo, min(w.z & ~3, kBig) + T_og,
                                             min(w.w & ~3, kBig) + T_os, (w.y & 255) + ord_off, s_thr[k + 1], m);
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) {
            if (!kChainTail && j == NB - 1) {
                sync->fin[0] = vo_p;
                sync->fin[1] = vg_p;
                sync->fin[2] = vs_p;
            }
            *v_final = j + 1;
            bar_arrive(&sync->bar_final[j]);
        }
    }

    if (aborted) {
        if (lane == 0) {
            a.counts[col] = 0;
            if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
            if (a.cost_fixed) a.cost_fixed[col] = kBig;
            atomicOr(a.err, STIXELS_ERR_TIMEOUT);
        }
        return;
    }
    // the partial minima (s_runv) are free now: the column's tail stages the
    // stixels there
    if constexpr (kChainTail) lead_column_end(ta, col, H, sync, s_bp, s_pd8, s_thr, s_div, s_runv, lane, vo_p, vg_p, vs_p);
}

// MINB: CTAs per SM the register allocation is sized for (8 warps x 2 CTAs
// and 16 warps x 1 CTA both leave 128 registers per thread, 8 x 3 leaves 85).
template <int NW, bool kStd, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) stixel_dp_kernel(DpArgs a, int ring, int slots, int window)
{
    extern __shared__ __align__(16) int32_t sm[];
    // a copy of the arguments in shared memory for the column's tail
    __shared__ DpArgs s_args;
    {
        const int* src = reinterpret_cast<const int*>(&a);
        int* dst = reinterpret_cast<int*>(&s_args);
        for (int i = threadIdx.x; i < (int)(sizeof(DpArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    // (dp_column's first barrier orders these stores before any read)
    dp_column<NW, kStd, true>(a, s_args, blockIdx.x, ring, slots, window, sm, 0);
}

// Persistent form: each CTA takes columns from a work list (one shared atomic
// counter, reset before the launch) until the list is empty.  The list is
// ordered longest column first, so the last columns to start are the short ones.
template <int NW, bool kStd, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
    stixel_dp_batch_kernel(const DpArgs* __restrict__ frames, const int2* __restrict__ items, int nitems,
                           int* counter, int ring, int slots, int window)
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
        dp_column<NW, kStd, false>(s_args, s_args, w.y, ring, slots, window, sm, w.y & 3);
        __syncthreads();
        // the next column initialises its barriers afresh
        SyncState* sync = dp_sync_state(sm, s_args.H, ring, slots);
        if (threadIdx.x < kMaxBlocks) bar_inval(&sync->bar_final[threadIdx.x]);
    }
}

// The bounded wait on a flag that nothing sets: it runs out after `limit`
// polls, records STIXELS_ERR_TIMEOUT and returns (how every DP wait ends when
// its partner stops), so the host sees a status and the context stays usable.
__global__ void __launch_bounds__(64) wait_selftest_kernel(uint32_t* err, int limit)
{
    __shared__ int flag, abort_flag;
    if (threadIdx.x == 0) {
        flag = 0;
        abort_flag = 0;
    }
    __syncthreads();
    if (threadIdx.x < 32 && !wait_geq(&flag, 1, &abort_flag, 32, limit) && threadIdx.x == 0)
        atomicOr(err, STIXELS_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_selftest(uint32_t* err, int limit, cudaStream_t st)
{
    if (limit < 1) return cudaErrorInvalidValue;
    wait_selftest_kernel<<<1, 64, 0, st>>>(err, limit);
    return cudaGetLastError();
}

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
template <int NW, bool kStd, int MINB>
bool* frame_flags() { static bool f[64] = {false}; return f; }
template <int NW, bool kStd, int MINB>
bool* batch_flags() { static bool f[64] = {false}; return f; }

// Partial minima per end row for columns of height H with `ring` chain
// buffers, `ctas` CTAs per SM: three (more warps share each end block's
// tiles, which the bound prunes newest first inside a window of two of the
// chain's blocks) where the shared memory has room, else two.
int pick_slots(int H, int ring, int ctas)
{
    const size_t per_cta = std::min<size_t>(227 * 1024, 228 * 1024 / ctas) - 2048;   // room for static + reserve
    return dp_smem_bytes(H, ring, 3) <= per_cta ? 3 : 2;
}

// The window of an end block's tiles (see dp_column), in chain blocks, by
// launch shape.  Pruning needs the newest tiles first, which packs a block's
// tile work into the window; measured (1024x440 / 2048x880 frames, 32 and 64
// frame batches):
//   - per frame, two columns per SM: window 2 with three partial minima
//     96.3 / 521 us against 100-102 / 658 us with no pruning;
//   - per frame, one column per SM (1024x440 at s = 7): 77.3 us against 73.7;
//   - batched: 13.1 K / 9.5 K frames/s against 13.3 K / 10.2 K with none.
// kNoPruning keeps every tile in start order, as the tiles become ready.
constexpr int kNoPruning = kMaxBlocks;
constexpr int kFrameWindow = 2;

template <int NW, bool kStd, int MINB>
cudaError_t launch_frame(const DpArgs& a, int ncols, cudaStream_t st)
{
    cudaError_t e = allow_smem(stixel_dp_kernel<NW, kStd, MINB>, frame_flags<NW, kStd, MINB>());
    if (e != cudaSuccess) return e;
    const bool prune = MINB >= 2;
    const int slots = prune ? pick_slots(a.H, kRingMax, MINB) : 2;
    // a programmatic dependent of the LUT kernel before it on the stream
    return launch_dependent(stixel_dp_kernel<NW, kStd, MINB>, dim3(ncols), dim3(NW * 32),
                            dp_smem_bytes(a.H, kRingMax, slots), st, a, (int)kRingMax, slots,
                            prune ? kFrameWindow : kNoPruning);
}

template <int NW, bool kStd, int MINB>
cudaError_t launch_batch(const DpArgs* frames, const int2* items, int nitems, int* counter, int grid, int maxH,
                         int ring, int ctas, cudaStream_t st)
{
    cudaError_t e = allow_smem(stixel_dp_batch_kernel<NW, kStd, MINB>, batch_flags<NW, kStd, MINB>());
    if (e != cudaSuccess) return e;
    (void)ctas;
    stixel_dp_batch_kernel<NW, kStd, MINB><<<grid, NW * 32, dp_smem_bytes(maxH, ring, 2), st>>>(
        frames, items, nitems, counter, ring, 2, kNoPruning);
    return cudaGetLastError();
}

bool standard_transitions(const ModelDev& m)
{
    return m.trans[1][1] >= kBig && m.trans[1][2] >= kBig && m.trans[2][2] >= kBig;
}

template <bool kStd>
cudaError_t launch_frame_shape(const DpArgs& a, int ncols, cudaStream_t st)
{
    // with no more columns than SMs, each column gets a whole SM: 16 warps
    // (15 bulk); otherwise two 8-warp CTAs share an SM
    if (ncols <= sm_count()) return launch_frame<16, kStd, 1>(a, ncols, st);
    return launch_frame<8, kStd, 2>(a, ncols, st);
}

template <bool kStd>
cudaError_t prepare_std()
{
    cudaError_t e = allow_smem(stixel_dp_batch_kernel<8, kStd, 2>, batch_flags<8, kStd, 2>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_batch_kernel<16, kStd, 1>, batch_flags<16, kStd, 1>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_batch_kernel<8, kStd, 3>, batch_flags<8, kStd, 3>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_kernel<8, kStd, 2>, frame_flags<8, kStd, 2>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_kernel<16, kStd, 1>, frame_flags<16, kStd, 1>());
    return e;
}

template <bool kStd>
cudaError_t launch_batch_shape(const DpArgs* f, const int2* it, int n, int* ctr, int warps, int grid, int ctas_per_sm,
                               int maxH, cudaStream_t st)
{
    // three 8-warp CTAs per SM fit the registers; a ring of two chain buffers
    // lets them fit the shared memory too (for heights up to about 450)
    if (warps == 16) return launch_batch<16, kStd, 1>(f, it, n, ctr, grid, maxH, kRingMax, 1, st);
    if (ctas_per_sm >= 3) return launch_batch<8, kStd, 3>(f, it, n, ctr, grid, maxH, 2, 3, st);
    return launch_batch<8, kStd, 2>(f, it, n, ctr, grid, maxH, kRingMax, 2, st);
}

}  // namespace

size_t dp_shared_bytes(int H) { return dp_smem_bytes(H, kRingMax, pick_slots(H, kRingMax, 2)); }

void dp_frame_args(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po, const FrameGeom& g,
                   const ModelDev& m, const RowsDev& r, const RealParams& rp, int32_t pixel_floor,
                   const stixels_output_t& out, uint32_t* err, DpArgs* a)
{
    a->pd = pd; a->pg = pg; a->ps = ps; a->po = po;
    a->H = g.H; a->P = g.P; a->F = m.dmax + 1;
    a->m = m; a->rows = r;
    a->stixels = out.stixels; a->counts = out.counts; a->cost = out.column_cost; a->cost_fixed = out.column_cost_fixed;
    a->cap = out.capacity;
    a->err = err;
    a->rp = rp;
    a->pixel_floor = pixel_floor;
}

cudaError_t launch_dp(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                      const FrameGeom& g, const ModelDev& m, const RowsDev& r, const RealParams& rp,
                      int32_t pixel_floor, const stixels_output_t& out, uint32_t* err, cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    if (g.H > STIXELS_MAX_HEIGHT) return cudaErrorInvalidValue;
    DpArgs a;
    dp_frame_args(pd, pg, ps, po, g, m, r, rp, pixel_floor, out, err, &a);
    return standard_transitions(m) ? launch_frame_shape<true>(a, g.ncols, st)
                                   : launch_frame_shape<false>(a, g.ncols, st);
}

cudaError_t prepare_dp_kernels()
{
    // attribute changes are not stream operations: do them before any capture
    cudaError_t e = prepare_std<true>();
    if (e == cudaSuccess) e = prepare_std<false>();
    if (e == cudaSuccess && sm_count() <= 0) e = cudaErrorInvalidDevice;
    return e;
}

cudaError_t launch_dp_batch(const DpArgs* d_frames, const int2* d_items, int nitems, int* d_counter, int maxH,
                            int warps, int ctas_per_sm, bool std_trans, int grid, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (maxH <= 0 || maxH > STIXELS_MAX_HEIGHT || grid <= 0) return cudaErrorInvalidValue;
    return std_trans ? launch_batch_shape<true>(d_frames, d_items, nitems, d_counter, warps, grid, ctas_per_sm, maxH, st)
                     : launch_batch_shape<false>(d_frames, d_items, nitems, d_counter, warps, grid, ctas_per_sm, maxH,
                                                 st);
}

}  // namespace stx
