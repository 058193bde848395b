// real_cost.cuh -- the cost of a solved column's segmentation in real
// arithmetic, for the DP kernels' epilogue.
//
// The DP (Eq. 5-6) decides on exact fixed-point costs: every per-pixel cost
// term and prior on a 2^-12 grid.  Those roundings are systematic (one K(f)
// per object disparity, one C_out, one sky K), so the fixed-point optimum of a
// column is off from the real-valued Eq. 4-6 cost by up to ~1.4e-5 relative.
// The column cost the library reports is therefore the cost of the chosen
// segmentation re-evaluated without the grid: per pixel Eq. 4,
//   min(C_out, K(f) + (d - f)^2 / (2 sigma^2)),
// with the object model f = the stixel's rounded mean, the ground model the
// unrounded ground line of the row, the sky model f = 0; plus, per stixel, the
// first-stixel / transition prior + BIC and the gravity, diving and ordering
// penalties (Sec. 3 constraints).  Per-pixel terms are FP32 (relative error
// of a few 1e-8 each); they and the priors are summed exactly in int64 fixed
// point at 2^-24 cost units (rounding each pixel by at most 3e-8), so the
// result does not depend on the order of the sum.  No FP64: on this part its
// latency is far above the FP32 and integer pipes'.
#pragma once

#include "internal.h"

namespace stx {

// The rounded mean f of stixel (b, k): floor((S + 8 n) / (16 n)) from the
// disparity prefix, by the multiply-high constants of n (div[n] = {M, s}),
// clamped to [0, dmax] as the DP's.
__device__ __forceinline__ int seg_mean_f(const int32_t* pd8, const uint2* div, int b, int k, int dmax)
{
    const uint2 dm = div[k - b + 1];
    return (int)min(__umulhi((uint32_t)(pd8[k + 1] - pd8[b]), dm.x) >> dm.y, (uint32_t)dmax);
}

// The per-f tables of a RealModelDev follow it in its allocation: k_obj[F],
// then inv_obj[F].  Addressing them from the struct's own address saves the
// dependent load of the pointers.
__device__ __forceinline__ const float* real_k_obj(const RealModelDev* rm)
{
    return reinterpret_cast<const float*>(rm + 1);
}

constexpr int kPreRows = 4;           // rows per lane whose tables are loaded in one go

// One lane's row tables for kPreRows rows (rows past the column repeat the
// last), loaded together so that their latency is paid once: the ground code
// gf, the line's offset rdg, K and 1 / (2 sigma^2).
struct RowTables {
    int gq[kPreRows];
    float gd[kPreRows], gk[kPreRows], gi[kPreRows];
};

// The row tables of rows 32 (jb + r dj) + lane, r < kPreRows.
__device__ __forceinline__ void load_rows(RowTables& t, const double* __restrict__ fg, int H, int lane, int jb, int dj)
{
    const int32_t* __restrict__ gf = rows_gf(fg, H);
    const float* __restrict__ rdg = rows_rdg(fg, H);
    const float* __restrict__ rkg = rows_rkg(fg, H);
    const float* __restrict__ rinv = rows_rinv(fg, H);
#pragma unroll
    for (int r = 0; r < kPreRows; ++r) {
        const int v = min(32 * (jb + r * dj) + lane, H - 1);
        t.gq[r] = __ldg(gf + v);
        t.gd[r] = __ldg(rdg + v);
        t.gk[r] = __ldg(rkg + v);
        t.gi[r] = __ldg(rinv + v);
    }
}

// The object K and 1 / (2 sigma^2) of every f (F <= 256), spread over a
// warp's registers (f = 32 j + lane), so that a lane can take any f's by
// shuffles instead of a memory round trip.
struct FTables {
    float k[8], inv[8];
};

__device__ __forceinline__ void load_ftables(FTables& t, const DpArgs& a, int lane)
{
    const float* __restrict__ k_obj = real_k_obj(a.rows.real_model);
    const float* __restrict__ inv_obj = k_obj + a.F;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int f = min(32 * j + lane, a.F - 1);
        t.k[j] = __ldg(k_obj + f);
        t.inv[j] = __ldg(inv_obj + f);
    }
}

// {K, 1 / (2 sigma^2)} of object disparity f from the FTables, by every lane
// of the warp together.
__device__ __forceinline__ float2 ftables_at(const FTables& t, int f)
{
    float2 r = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float k = __shfl_sync(0xffffffffu, t.k[j], f & 31);
        const float i = __shfl_sync(0xffffffffu, t.inv[j], f & 31);
        if ((f >> 5) == j) r = make_float2(k, i);
    }
    return r;
}

// The report in two parts, over the stixel list scr[i] = b << 13 | k << 2 |
// class of stixel i (bottom-up rows b..k), bottom -> top, n entries, in
// shared memory with room for 4 H words; pd8[v] = PD[v] + 8 v for v = 0..H
// and div the rounded-mean constants (shared memory); H the rows covered.
// Sums are in units of 2^-24 (kReportUnits).  The priors and the outlier /
// sky constants come from the kernel arguments (a.rp); the gravity / diving /
// ordering decisions are the DP's own integer tests, which the host derived
// from the same comparisons on the unrounded ground line.
//
// report_stixels (one warp, every lane; lane l stixels l, l + 32, ...): each
// stixel's prior, summed into the lane's return value, and the constants of
// its pixel cost, staged in scr[H..4H) for report_rows.  kinv(f, valid)
// gives {K, 1 / (2 sigma^2)} of object disparity f (called by every lane
// together); thr(b) the {fhi, flo} gravity / diving thresholds of row b.
template <class KInv, class Thr>
__device__ __forceinline__ long long report_stixels(int32_t* scr, int n, const int32_t* pd8, const uint2* div,
                                                    const DpArgs& a, int H, int lane, KInv kinv, Thr thr)
{
    const int dmax = a.m.dmax, ord_off = a.m.ord_off;
    const RealParams& rp = a.rp;
    float* s_k = reinterpret_cast<float*>(scr + H);      // K of the stixel's model (object, sky)
    float* s_inv = s_k + H;                              // 1 / (2 sigma^2)
    int32_t* s_m16 = scr + 3 * H;                        // 16 f of its model (sky 0)
    long long acc = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool valid = i < n;
        const int w = valid ? scr[i] : 0;
        const int b = w >> 13, k = (w >> 2) & 2047, c = w & 3;
        const int f = seg_mean_f(pd8, div, b, k, dmax);
        const float2 ki = kinv(f, valid);
        if (!valid) continue;
        const int wp = i > 0 ? scr[i - 1] : 0;
        const int pc = wp & 3;
        long long pr;
        if (i == 0) {
            pr = rp.first[c];
        } else {
            pr = rp.trans[c][pc];
            if (c == 0 && pc == 1) {
                const int2 t = thr(b);
                if (f > t.x) pr += rp.pen_grav;
                if (f < t.y) pr += rp.pen_div;
            }
            if (c == 0 && pc == 0 && f > seg_mean_f(pd8, div, wp >> 13, (wp >> 2) & 2047, dmax) + ord_off)
                pr += rp.pen_ord;
        }
        acc += pr;
        s_k[i] = c == 0 ? ki.x : rp.k_sky;
        s_inv[i] = c == 0 ? ki.y : rp.inv_sky;
        s_m16[i] = c == 0 ? 16 * f : 0;
    }
    return acc;
}

// report_rows (one warp): Eq. 4 per pixel, under the model of the stixel that
// holds it, for the rows 32 j + lane of the row blocks j = j0, j0 + dj, ...;
// returns the lane's sum.  Each lane walks the list once, its rows ascending;
// its row tables come kPreRows at a time, all in flight (the first group,
// rows of blocks j0 + r dj, may come preloaded).
__device__ __forceinline__ long long report_rows(const int32_t* scr, int n, const int32_t* pd8, const DpArgs& a,
                                                 int H, int lane, int j0, int dj, const RowTables* first)
{
    const float* s_k = reinterpret_cast<const float*>(scr + H);
    const float* s_inv = s_k + H;
    const int32_t* s_m16 = scr + 3 * H;
    const float c_out = a.rp.c_out;
    long long acc = 0;
    int si = 0;
    for (int jb = j0; 32 * jb < H; jb += kPreRows * dj) {
        RowTables t;
        if (jb == j0 && first) t = *first;
        else load_rows(t, a.rows.fg, H, lane, jb, dj);
#pragma unroll
        for (int r = 0; r < kPreRows; ++r) {
            const int v = 32 * (jb + r * dj) + lane;
            if (v < H) {
                while (si < n - 1 && ((scr[si] >> 2) & 2047) < v) ++si;   // the stixel of row v
                const int c = scr[si] & 3;
                const int q = pd8[v + 1] - pd8[v] - 8;
                float dpx, K, iv;
                if (c == 1) {
                    // (q - gf) / 16 is exact; rdg = f_g - gf / 16 is below 1/16
                    dpx = (float)(q - t.gq[r]) * 0.0625f - t.gd[r];
                    K = t.gk[r];
                    iv = t.gi[r];
                } else {
                    dpx = (float)(q - s_m16[si]) * 0.0625f;
                    K = s_k[si];
                    iv = s_inv[si];
                }
                // a pixel costs at most C_out (< 2^7 units), so this fits int32
                acc += __float2int_rn(fminf(c_out, K + dpx * dpx * iv) * kReportUnits);
            }
        }
    }
    return acc;
}

__device__ __forceinline__ long long warp_sum64(long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// The whole report by one warp, reading its tables from global memory (every
// lane returns the cost in 2^-24 units); thr(b) as for report_stixels.
template <class Thr>
__device__ __forceinline__ long long real_segmentation_cost(int32_t* scr, int n, const int32_t* pd8, const uint2* div,
                                                            const DpArgs& a, int H, int lane, Thr thr)
{
    const float* __restrict__ k_obj = real_k_obj(a.rows.real_model);
    const float* __restrict__ inv_obj = k_obj + a.F;
    auto kinv = [&](int f, bool valid) {
        return valid ? make_float2(__ldg(k_obj + f), __ldg(inv_obj + f)) : make_float2(0.f, 0.f);
    };
    long long acc = report_stixels(scr, n, pd8, div, a, H, lane, kinv, thr);
    __syncwarp();
    acc += report_rows(scr, n, pd8, a, H, lane, 0, 1, nullptr);
    return warp_sum64(acc);
}

}  // namespace stx
