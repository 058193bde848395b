// internal.h -- shared declarations of the stixel library's host code and kernels.
#pragma once

#include <stdint.h>

#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "stixels.h"

namespace stx {

// Programmatic dependent launch: a kernel launched with launch_dependent may
// be scheduled while the one before it on the stream still runs (once every
// CTA of that one has started or called grid_dependents_may_launch); it must
// call grid_dependency_wait before it reads what the earlier kernel writes or
// writes what that one reads.  Both are no-ops for a kernel launched plainly.
#ifdef __CUDACC__
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_may_launch() { asm volatile("griddepcontrol.launch_dependents;"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
#endif

// Fixed-point cost arithmetic.  Costs are int32 in units of 2^-14; every
// per-pixel term and every prior is a multiple of 4 (i.e. on the 2^-12 grid),
// so the two low bits of a candidate cost are free to carry the code of the
// previous class (0 object, 1 ground, 2 sky, 3 none = first stixel).  A
// packed value (cost + code) then orders candidates by (cost, code).
constexpr int32_t kUnitsPerCost = 16384;         // 2^14
constexpr int32_t kBig = 1 << 29;                // infeasible / forbidden
constexpr int32_t kFiniteBudget = 1 << 28;       // |finite cost| bound checked by the host
constexpr int32_t kNoneCode = 3;

// floor(x / (16 n)) for 0 <= x < 2^31 via a multiply-high: M = ceil(2^(32+s) / d),
// s = floor(log2 d), d = 16 n (M = 2^31, s - 1 when d is a power of two).
// The constants for n = 1 .. STIXELS_MAX_HEIGHT are built at compile time;
// each DP kernel's translation unit holds one copy in device memory and every
// CTA copies the ones its column height needs into shared memory.
struct alignas(8) DivMagic {
    uint32_t m, s;
};
struct DivTable {
    DivMagic v[STIXELS_MAX_HEIGHT + 1];
};
constexpr DivTable make_div_table()
{
    DivTable t{};
    for (int n = 1; n <= STIXELS_MAX_HEIGHT; ++n) {
        const uint32_t d = 16u * (uint32_t)n;
        int s = 0;
        while ((d >> (s + 1)) != 0) ++s;
        if ((d & (d - 1)) == 0) {
            t.v[n] = DivMagic{1u << 31, (uint32_t)(s - 1)};
        } else {
            const unsigned long long num = 1ull << (32 + s);
            t.v[n] = DivMagic{(uint32_t)((num + d - 1) / d), (uint32_t)s};
        }
    }
    return t;
}

// The priors without the cost grid (prior + BIC, penalties) and the outlier
// and sky constants, for the cost report: kernel arguments, so that the report
// reads no memory for them.  The report sums in int64 fixed point with
// kReportUnits per cost unit (a prior's rounding: <= 3e-8), since FP64 is far
// slower than the FP32 / integer pipes on this part.
constexpr float kReportUnits = 16777216.0f;       // 2^24
constexpr long long kReportInf = 1ll << 60;       // a forbidden prior (never on a solved path)
struct RealParams {
    long long first[3];      // first-stixel prior + BIC, per class
    long long trans[3][3];   // [above][below] transition prior + BIC
    long long pen_grav, pen_div, pen_ord;
    float c_out, k_sky, inv_sky, pad;
};

// The model without the fixed-point grid, resident on the device: what the
// DP kernels' epilogue needs to report a solved segmentation's cost in real
// arithmetic (Eq. 3-4 per pixel in FP32, sums in int64 fixed point).  The
// struct is followed in the same allocation by float k_obj[dmax + 1] (object
// K at integer f), float inv_obj[dmax + 1] (1 / (2 sigma^2)) and, for the
// ground estimate, rkg_tab.
struct RealModelDev {
    RealParams rp;           // the priors and constants (copied into each frame's DP arguments)
    double eps_g, eps_d;     // gravity / diving tolerances (px): an estimated line's thresholds
    float inv_ground;        // 1 / (2 sigma_g^2): an estimated line's rows
    int32_t dmax;
    const float* rkg_tab;    // ground estimate only: [256 dmax + 1] unrounded ground K at f = c / 256
};

// Per-handle model, resident on the device (the "offline" LUTs of Sec. 3.4)
// plus the scalars every kernel needs.  Passed to kernels by value.
struct ModelDev {
    int32_t dmax;            // F = dmax + 1 object disparities
    int32_t emax;            // 16 * dmax: largest tabulated Q4 residual
    int32_t c_out;           // outlier branch of Eq. 4
    int32_t k_sky;           // K of the sky model (f = 0)
    int32_t first[3];        // first-stixel prior + BIC, per class
    int32_t trans[3][3];     // [above][below] transition prior + BIC
    int32_t pen_grav, pen_div, pen_ord;
    int32_t ord_off;         // ordering penalty iff f_above > f_below + ord_off (floor of eps_order)
    // saturation residual per class: for e >= esat, K + G[e] >= C_out for every K
    // of that class, so min(C_out, K + G[min(e, esat)]) equals the unclamped cost
    int32_t esat_obj, esat_sky;
    const int32_t* k_obj;    // [dmax + 1]
    const int32_t* g_obj;    // [emax + 1]
    const int32_t* g_sky;    // [emax + 1]
    int32_t var_sigma;       // 1: g_obj is [dmax + 1][emax + 1] (one residual row per f)
    int32_t int_grid;        // 1: reduced disparities are whole pixels (multiples of 16 in Q4)
    const int32_t* lut_cost; // int_grid only: [dmax + 1][dmax + 1], object cost of (f, d)
    const int32_t* kg_tab;   // ground estimate only: [256 dmax + 1] ground K at f = c / 256 (clamped)
};

// Per-row tables of one height (a handle's camera line, or one frame's
// estimated line), one device block; v = bottom-up row:
//   double fg[H]   the ground model's disparity f_g(v) (Sec. 3.1), unrounded
//   int32  kg[H]   the ground K on the cost grid
//   int32  thr[H]  gravity / diving thresholds on the object's f, as int16
//                  halves: penalty iff f > fhi (low), iff f < flo (high)
//   int32  gf[H]   floor(16 f_g): the Q4 code at or below the line
//   int32  goff[H] offset of the row's residual window in gpool
//   float  rkg[H]  the ground K unrounded (cost report)
//   float  rinv[H] 1 / (2 sigma_g^2) (cost report)
//   float  rdg[H]  f_g - gf / 16, in [0, 1/16) (cost report)
// The ground residual of a pixel with Q4 code q, (q / 16 - f_g)^2 / (2
// sigma_g^2) on the cost grid, is gpool[goff[v] + q - (gf[v] - ER)] for the
// gw = 2 ER + 2 codes q of the row's window; every code outside it is at
// least ER / 16 px from the line, where the pixel costs C_out.  A camera
// line's windows (one per row) follow the arrays in the same block; an
// estimated line's disparities are multiples of 1/256 px, so its rows share
// 16 windows built at create time.
struct RowsDev {
    const double* fg;                 // start of the block
    const RealModelDev* real_model;   // the handle's model without the grid (cost report)
    const int32_t* gpool;             // ground residual windows
    int32_t gw;                       // codes per window, 2 ER + 2
    int32_t gn;                       // words of gpool
};
__host__ __device__ inline size_t rows_arrays_bytes(int H) { return ((size_t)H * 36 + 15) / 16 * 16; }
__host__ __device__ inline const int32_t* rows_kg(const double* fg, int H)
{
    return reinterpret_cast<const int32_t*>(fg + H);
}
__host__ __device__ inline const int32_t* rows_thr(const double* fg, int H) { return rows_kg(fg, H) + H; }
__host__ __device__ inline const int32_t* rows_gf(const double* fg, int H) { return rows_kg(fg, H) + 2 * H; }
__host__ __device__ inline const int32_t* rows_goff(const double* fg, int H) { return rows_kg(fg, H) + 3 * H; }
__host__ __device__ inline const float* rows_rkg(const double* fg, int H)
{
    return reinterpret_cast<const float*>(rows_kg(fg, H) + 4 * H);
}
__host__ __device__ inline const float* rows_rinv(const double* fg, int H) { return rows_rkg(fg, H) + H; }
__host__ __device__ inline const float* rows_rdg(const double* fg, int H) { return rows_rkg(fg, H) + 2 * H; }
// the packed thresholds for a ground disparity fg: penalty iff 16 f > 16 (fg +
// eps_g), i.e. f > floor(fg + eps_g); iff f < fg - eps_d, i.e. f < ceil(fg -
// eps_d); clamped to [-1, 256], which keeps every comparison with f in [0, 255]
__host__ __device__ inline int32_t pack_thresholds(double fg, double eps_g, double eps_d)
{
    const double hi = floor(fg + eps_g), lo = ceil(fg - eps_d);
    const int fhi = hi < -1.0 ? -1 : (hi > 256.0 ? 256 : (int)hi);
    const int flo = lo < -1.0 ? -1 : (lo > 256.0 ? 256 : (int)lo);
    return (int32_t)((uint32_t)(fhi & 0xffff) | ((uint32_t)flo << 16));
}

struct FrameGeom {
    int H, W, s, ncols;
    int P;                   // LUT pitch (int32 elements), multiple of 4, >= H + 1
};

inline int lut_pitch(int H) { return ((H + 1) + 3) & ~3; }

// One frame's arguments for the reduction kernel (batch table entry).
struct ReduceArgs {
    const float* disp;
    int H, W, ncols, dmax;
    int16_t* q;
};

// One frame's arguments for the LUT kernel.
struct LutArgs {
    const int16_t* q;
    int H, P, F;
    ModelDev m;
    RowsDev rows;
    int32_t* pd;
    int32_t* pg;
    int32_t* ps;
    int32_t* po;
    // 1: write only the object rows f that a stixel of the column can have as
    // its rounded mean, round(min q / 16) .. round(max q / 16) (the mean of a
    // run of codes lies between their extremes); the DP reads no other row
    int32_t range_only;
    int32_t rows_per_cta;       // LUT rows per CTA (lut_rows_per_cta)
};

// One frame's arguments for the DP kernel (per-frame launch or batch table entry).
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
    RealParams rp;
    int32_t pixel_floor;     // no object pixel costs less, at any f (2^-14 units; the DP's tile bound)
};

// What the scratch-free entry point needs from a prepared handle.
struct HandleView {
    int device;
    ModelDev model;
    RowsDev rows;
    RealParams rp;              // the cost report's priors and constants
    int32_t pixel_floor;        // the model's least object pixel cost (DpArgs::pixel_floor)
    uint32_t* err;
    int stixel_width, capacity;
    int reduce_mode;            // reduce_code of the params: bit 0 mean, bit 1 whole-pixel grid
    int ground_estimate;        // the handle estimates its ground per frame
    int global_map;             // the handle solves the global MAP
    const int32_t* est_pool;    // ground estimate: the residual windows of estimated lines
    int est_gw;                 // their codes per window
};
int handle_view(stixels_t h, int H, HandleView* v);
// stixels status for a CUDA error, remembering its text for stixels_last_cuda_error()
int status_from_cuda(cudaError_t e);
// The reduction kernels' mode: bit 0 = mean (else median), bit 1 = round to whole pixels.
inline int reduce_code(const stixels_params_t& p) { return (p.reduce_mode & 1) | ((p.pixel_grid & 1) << 1); }
const char* t_last_cuda_error_string();
int handle_prepare(stixels_t h, int H, HandleView* v);
int sm_count();

// ---- kernel launchers (kernels_*.cu); all return cudaGetLastError() ----
cudaError_t launch_reduce(const float* disp, const FrameGeom& g, int dmax, int mode, int16_t* q,
                          cudaStream_t st);
// range_only: see LutArgs (the library's own pipelines); 0 writes every row.
cudaError_t launch_luts(const int16_t* q, const FrameGeom& g, const ModelDev& m, const RowsDev& r,
                        int32_t* pd, int32_t* pg, int32_t* ps, int32_t* po, cudaStream_t st, int range_only = 0);
size_t lut_shared_bytes(int H, const ModelDev& m);
// LUT rows per CTA: 48 where only the code range is written with the
// default model (fewer CTAs that skip every row), else 32
int lut_rows_per_cta(const ModelDev& m, int range_only);
int lut_row_groups(int F, int rows_per_cta);
cudaError_t launch_luts_batch(const LutArgs* d_frames, const int2* d_items, int nitems, int max_groups,
                              size_t smem, cudaStream_t st);
cudaError_t launch_reduce_batch(const ReduceArgs* d_frames, const int4* d_tiles, int ntiles, int s, int mode,
                                cudaStream_t st);
cudaError_t launch_dp(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                      const FrameGeom& g, const ModelDev& m, const RowsDev& r, const RealParams& rp,
                      int32_t pixel_floor, const stixels_output_t& out, uint32_t* err, cudaStream_t st);
void dp_frame_args(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po, const FrameGeom& g,
                   const ModelDev& m, const RowsDev& r, const RealParams& rp, int32_t pixel_floor,
                   const stixels_output_t& out, uint32_t* err, DpArgs* a);
size_t dp_shared_bytes(int H);
// ---- batch planning shared by the batched mode and the server (batch.cu) ----
// One frame's device buffers for a pipeline run.
struct FrameJob {
    HandleView view;
    FrameGeom g;
    const float* in;
    int16_t* q;
    int32_t *pd, *pg, *ps, *po;
    char* ground_work;          // ground estimate: the frame's v-disparity work and row tables
    void* map_scratch;          // global MAP: the DP's scratch
    stixels_output_t out;
};
// Bytes of intermediates (q, PD, PG, PS, PO, and the ground-estimate work and
// global-MAP scratch when the view asks for them) a frame needs, and their
// carving from one 256-byte-aligned block.
size_t frame_work_bytes(const FrameGeom& g, const HandleView& v);
void frame_work_carve(FrameJob* job, char* base);
struct ReduceGroup {            // frames sharing stixel width and reduction mode
    int s, mode;
    size_t tiles_off;           // offset of its int4 tiles in the table block
    int ntiles;
};
// Host image of the argument tables and work lists of a set of frames.
struct BatchTables {
    std::vector<char> host;
    size_t o_red = 0, o_lut = 0, o_dp = 0, o_li = 0, o_di = 0, o_cnt = 0;
    std::vector<ReduceGroup> groups;
    int nitems = 0, max_groups = 0, maxH = 0;
    int nlut = 0;               // LUT work items (every frame's columns)
    size_t lut_smem = 0;
    bool std_trans = true;
    // frames whose ground line is estimated: their arguments (GroundArgs per
    // frame) and (frame, row block), (frame, horizon block) items; ground_ok
    // false when one of them has no estimate windows
    size_t o_ga = 0, o_gr = 0, o_gv = 0;
    int ngr = 0, ngv = 0;
    size_t ground_smem = 0;
    bool ground_ok = true;
    // frames solved by the global MAP (one launch over their columns): their
    // scratch rows (MapScratch per frame) and (frame, column) items
    size_t o_ms = 0, o_mi = 0;
    int nmap = 0;                     // global-MAP items
    size_t map_smem = 0;
    std::vector<FrameJob> jobs;       // the frames, for those launches
};
void plan_tables(const std::vector<FrameJob>& jobs, BatchTables* t);
// One frame through the per-frame kernels (the launches of stixels_compute)
// on the job's own buffers.
cudaError_t launch_frame_job(const FrameJob& f, cudaStream_t st);
// Launches all stages for tables already copied to d_tab (counter reset included).
cudaError_t enqueue_tables(const BatchTables& t, char* d_tab, int dp_warps, int dp_ctas_per_sm, cudaStream_t st);

// The frame's ground line from its v-disparity (kernels_ground.cu): work bytes
// for height H (gw: codes per residual window), and the launch (cam = the
// camera's rows, kept when nothing votes; est_pool / est_gw = the handle's
// residual windows of estimated lines, est_gw == cam.gw; frame_rows receives
// the frame's tables inside `work`; line, if not null, receives {k, horizon
// row, votes} on the device).
size_t ground_work_bytes(int H, int dmax, int gw);
// The ground estimate's int32 votes stay below 289 ncols H (the smoothing
// kernel's weight times every column of every row).
inline bool ground_size_ok(const FrameGeom& g) { return (int64_t)g.ncols * g.H <= 7000000; }
// The frame's row tables that launch_ground writes inside `work`.
RowsDev ground_frame_rows(const FrameGeom& g, int dmax, const RowsDev& cam, int est_gw, char* work);
cudaError_t prepare_ground_kernels();
// One frame's ground-estimate arguments (the per-frame launch's, for the
// batch kernels' table rows): false when the handle has no estimated-line
// windows matching its camera's.
struct GroundArgs {
    const int16_t* q;
    int H, ncols, dmax, gw;
    int32_t* smooth;
    unsigned long long* best;
    const int32_t* kg_tab;
    RowsDev cam;
    const RealModelDev* rm;
    const int32_t* est_pool;
    double* rows;
    int32_t* pool;
    int32_t* line;
    int nvote;                  // the frame's vote blocks
};
bool ground_args(const int16_t* q, const FrameGeom& g, const ModelDev& m, const RowsDev& cam, const int32_t* est_pool,
                 int est_gw, char* work, int32_t* line, GroundArgs* a);
int ground_row_blocks(int H);        // v-disparity CTAs of a frame (two image rows each)
int ground_horizon_blocks(int H);    // vote CTAs of a frame per slope (128 horizons each)
size_t ground_vdisp_smem(int dmax);
// Batch form: one v-disparity launch over (frame, row block) items, then one
// vote launch over (frame, horizon block) items x 256 slopes.
cudaError_t launch_ground_batch(const GroundArgs* d_args, const int2* d_row_items, int nrow_items,
                                const int2* d_vote_items, int nvote_items, size_t vdisp_smem, cudaStream_t st);
cudaError_t launch_ground(const int16_t* q, const FrameGeom& g, const ModelDev& m, RowsDev cam,
                          const int32_t* est_pool, int est_gw, char* work, RowsDev* frame_rows, int32_t* line,
                          cudaStream_t st);

// The global-MAP DP (kernels_dp_map.cu): scratch bytes for a frame, and the launch.
size_t map_scratch_bytes(int H, int ncols, int F);
// One CTA whose bounded wait (the DP kernels' own) runs out after `limit` polls.
cudaError_t launch_wait_selftest(uint32_t* err, int limit, cudaStream_t st);
// Whether a column of height H with F object disparities fits the global-MAP
// kernel's shared memory (226 KB of dynamic shared memory per CTA; every
// column the library takes, up to 2048 rows at dmax 255, does).
bool map_fits(int H, int F);
// Sets the global-MAP kernel's shared-memory attribute (call outside stream capture).
cudaError_t prepare_map_kernel();
cudaError_t launch_dp_map(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                          const FrameGeom& g, const ModelDev& m, const RowsDev& r, const RealParams& rp,
                          int32_t pixel_floor, const stixels_output_t& out, uint32_t* err, void* scratch,
                          cudaStream_t st);
// A frame's global-MAP scratch (map_scratch_bytes at `scratch`): object
// states [ncols][H][F], ground / sky states [ncols][2][H], rows of M.
struct MapScratch {
    int32_t* keyo;
    int32_t* kgs;
    int32_t* mv;
};
MapScratch map_scratch_carve(void* scratch, int H, int ncols, int F);
// Dynamic shared memory of one global-MAP CTA for a column of height H.
size_t map_smem_bytes(int H, int F);
// Batch form: one CTA per (frame, column) item; frames[i] and scratch[i]
// describe frame i; smem = the largest map_smem_bytes of the frames.
cudaError_t launch_dp_map_batch(const DpArgs* d_frames, const MapScratch* d_scratch, const int2* d_items, int nitems,
                                size_t smem, cudaStream_t st);

// Sets the DP kernels' shared-memory attributes (call outside stream capture).
cudaError_t prepare_dp_kernels();
// Persistent DP over a work list of (frame, column) items; *d_counter must be 0.
cudaError_t launch_dp_batch(const DpArgs* d_frames, const int2* d_items, int nitems, int* d_counter, int maxH,
                            int warps, int ctas_per_sm, bool std_trans, int grid, cudaStream_t st);

}  // namespace stx
