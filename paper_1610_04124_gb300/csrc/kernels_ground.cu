// kernels_ground.cu -- the frame's ground line from its v-disparity (the step
// before the path: the paper takes the ground slope and horizon as known for
// every image, Sec. 3).
//
// On the 1/16-px grid of the reduced codes (image row r = H-1-v):
//   hist[r][e]  columns whose code at row r is e, for e in [16, 16 dmax]
//               (codes below 1 px -- sky, invalid pixels -- carry no ground);
//   S[r][e]     sum over |t| <= 16 of (17 - |t|) hist[r][e + t], a triangular
//               kernel of half-width 1 px so that noisy ground still votes;
//   line (k, h) code (k (r - h) + 8) >> 4 at rows r > h: slope k / 256 px of
//               disparity per image row (k = 1..256), horizon at image row h;
//   votes(k, h) sum of S[r][code] over the rows r > h with code in [16, 16 dmax];
// the line with the most votes wins, ties to the smaller k, then the smaller h.
// The line itself, f_g = k (r - h) / 256 px at image row r (not its Q4
// codes: those only index the vote), replaces the camera's ground line for
// the frame; the ground K of each row comes from a create-time table over
// the disparities c / 256.  With no vote at all the camera's line is kept.
//
// Kernels: one CTA per two image rows builds their histograms in shared
// memory, smooths them (the triangle as a box of 17 codes applied twice) and
// stores S code-major (S[e][r], rows padded to a multiple of two), so that
// for a fixed slope k and row offset j = r - h the code is the same for every
// horizon h and a warp over 32 consecutive h reads 32 consecutive words.  A
// vote CTA takes one k and 128 horizons (four per lane, so that one address
// serves four loads); its 8 warps split the offsets, 32 loads in flight
// each, and a 64-bit atomic max over (votes, 256 - k,
// 65535 - h) picks the winner whatever the order; the last vote CTA to
// finish writes the frame's row tables.
#include "internal.h"

namespace stx {
namespace {

constexpr int kVdispRows = 2;   // image rows per histogram CTA
constexpr int kVoteM = 4;              // horizons per lane, 32 apart
constexpr int kVoteH = 32 * kVoteM;    // horizons per vote CTA
constexpr int kVoteWarps = 8;          // warps per vote CTA, each over every eighth run of 8 offsets

// rows of the code-major table: the image height rounded up to kVdispRows
__host__ __device__ inline int ground_pitch(int H) { return (H + kVdispRows - 1) / kVdispRows * kVdispRows; }
// words per histogram row in shared memory: the E codes, then zeros far
// enough for the last run of 8 codes to read 24 words past its end, in whole
// 16-byte words
__host__ __device__ inline int vdisp_pitch(int E) { return (E + 23 + 3) / 4 * 4; }

// per two image rows (row block rb): histograms of the codes, smoothed,
// stored code-major
__device__ __forceinline__ void vdisp_rows(const int16_t* __restrict__ q, int H, int ncols, int dmax,
                                           int32_t* __restrict__ smooth, unsigned long long* __restrict__ best,
                                           const int rb)
{
    // the vote kernel that follows on the stream starts from no winner and no
    // finished block
    if (rb == 0 && threadIdx.x == 0) {
        best[0] = 0ull;
        best[1] = 0ull;
    }
    // s_h[i][x]: codes below 16 are never counted and the words from E on stay
    // zero, so every window below reads zeros outside [16, E)
    extern __shared__ __align__(16) int32_t s_h[];
    const int E = 16 * dmax + 1, P = vdisp_pitch(E), Hp = ground_pitch(H);
    const int r0 = rb * kVdispRows;
    for (int x = threadIdx.x; x < kVdispRows * P; x += blockDim.x) s_h[x] = 0;
    __syncthreads();
    // four codes' loads in flight per thread, then their counts
    for (int x0 = threadIdx.x; x0 < kVdispRows * ncols; x0 += 4 * blockDim.x) {
        int code[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = x0 + u * blockDim.x;
            const int c = x / kVdispRows, i = x % kVdispRows, r = r0 + i;
            code[u] = (x < kVdispRows * ncols && r < H) ? q[(size_t)c * H + (H - 1 - r)] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (code[u] >= 16 && code[u] < E) atomicAdd(&s_h[((x0 + u * blockDim.x) % kVdispRows) * P + code[u]], 1);
    }
    __syncthreads();
    // The triangle 17 - |t| (|t| <= 16) is a box of 17 codes convolved with
    // itself: B[y] = sum of hist over [y - 8, y + 8], S[e] = sum of B over
    // [e - 8, e + 8].  A thread takes 8 consecutive codes e0..e0+7 and slides
    // both boxes over the 40 words hist[e0 - 16 .. e0 + 23].
    const int G = (E - 16 + 7) / 8;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const int e0 = 16 + 8 * g;
        int32_t out[kVdispRows][8];
        static_assert(kVdispRows == 2, "one 8-byte store per code below");
#pragma unroll
        for (int i = 0; i < kVdispRows; ++i) {
            const int32_t* hp = s_h + i * P + 8 * g;   // code e0 - 16, 16-byte aligned
            int32_t hv[40];
#pragma unroll
            for (int m = 0; m < 40; m += 4) {
                const int4 x = *reinterpret_cast<const int4*>(hp + m);
                hv[m] = x.x;
                hv[m + 1] = x.y;
                hv[m + 2] = x.z;
                hv[m + 3] = x.w;
            }
            int32_t bx[24];   // bx[x] = B[e0 - 8 + x]
            int32_t acc = 0;
#pragma unroll
            for (int m = 0; m <= 16; ++m) acc += hv[m];
            bx[0] = acc;
#pragma unroll
            for (int x = 0; x < 23; ++x) {
                acc += hv[x + 17] - hv[x];
                bx[x + 1] = acc;
            }
            acc = 0;
#pragma unroll
            for (int m = 0; m <= 16; ++m) acc += bx[m];
            out[i][0] = acc;
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                acc += bx[o + 17] - bx[o];
                out[i][o + 1] = acc;
            }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o)
            if (e0 + o < E)
                *reinterpret_cast<int2*>(smooth + (size_t)(e0 + o) * Hp + r0) = make_int2(out[0][o], out[1][o]);
    }
    // codes below 16 carry no ground
    for (int e = threadIdx.x; e < 16; e += blockDim.x)
        *reinterpret_cast<int2*>(smooth + (size_t)e * Hp + r0) = make_int2(0, 0);
}

__global__ void __launch_bounds__(256) vdisp_kernel(const int16_t* __restrict__ q, int H, int ncols, int dmax,
                                                    int32_t* __restrict__ smooth, unsigned long long* __restrict__ best)
{
    vdisp_rows(q, H, ncols, dmax, smooth, best, blockIdx.x);
}

// the frame's row tables (RowsDev) from the winning line, or the camera's
// when nothing voted.  The line's ground disparity k (r - h) / 256 is a
// multiple of 1/256 px, so its K comes from the create-time tables over those
// disparities (clamped to [0, 256 dmax]: K depends on f only through its clamp
// to [0, d_range]), its gravity / diving thresholds follow from it in FP64,
// and its rows share the 16 residual windows of the create-time pool (one per
// phase x & 15 of 16 f_g = x / 16), copied into the frame's pool; the camera's
// own windows (as many codes each: the handle builds both with one reach) are
// copied instead when nothing voted.
__device__ __noinline__ void write_ground_rows(unsigned long long key, int H, int dmax,
                                               const int32_t* __restrict__ kg_tab, const RowsDev& cam,
                                               const RealModelDev* __restrict__ rm,
                                               const int32_t* __restrict__ est_pool, int gw,
                                               double* __restrict__ rows, int32_t* __restrict__ pool,
                                               int32_t* __restrict__ line)
{
    const int votes = (int)(key >> 32);
    const int k = 256 - (int)((key >> 16) & 0xffff);
    const int h = 65535 - (int)(key & 0xffff);
    const int cmax = 256 * dmax;
    int32_t* kg = reinterpret_cast<int32_t*>(rows + H);
    int32_t* thr = kg + H;
    int32_t* gf = kg + 2 * H;
    int32_t* goff = kg + 3 * H;
    float* rkg = reinterpret_cast<float*>(kg + 4 * H);
    float* rinv = rkg + H;
    float* rdg = rkg + 2 * H;
    const double* cfg = cam.fg;
    for (int v = threadIdx.x; v < H; v += blockDim.x) {
        if (votes > 0) {
            const int x = k * (H - 1 - v - h);
            const int c = min(max(x, 0), cmax);
            const double f = (double)k * (double)(H - 1 - v - h) / 256.0;
            rows[v] = f;
            kg[v] = kg_tab[c];
            thr[v] = pack_thresholds(f, rm->eps_g, rm->eps_d);
            gf[v] = x >> 4;                              // floor(x / 16)
            goff[v] = (x & 15) * gw;
            rkg[v] = rm->rkg_tab[c];
            rinv[v] = rm->inv_ground;
            rdg[v] = (float)(x & 15) * (1.0f / 256.0f);
        } else {
            rows[v] = cfg[v];
            kg[v] = rows_kg(cfg, H)[v];
            thr[v] = rows_thr(cfg, H)[v];
            gf[v] = rows_gf(cfg, H)[v];
            goff[v] = rows_goff(cfg, H)[v];
            rkg[v] = rows_rkg(cfg, H)[v];
            rinv[v] = rows_rinv(cfg, H)[v];
            rdg[v] = rows_rdg(cfg, H)[v];
        }
    }
    const int n = votes > 0 ? 16 * gw : H * gw;
    const int32_t* src = votes > 0 ? est_pool : cam.gpool;
    for (int i = threadIdx.x; i < n; i += blockDim.x) pool[i] = src[i];
    if (threadIdx.x == 0 && line) {
        line[0] = k;
        line[1] = h;
        line[2] = votes;
    }
}

// one thread per four candidates and run of offsets: k = blockIdx.y + 1,
// h = blockIdx.x * kVoteH + lane + 32 m (m < kVoteM); warp w sums the offsets
// j in runs of 8 starting at j_lo + 8 w, every 8 kVoteWarps, and the block
// adds the warps' sums.  One address per offset serves the four horizons.
// best[0] is the running winner, best[1] counts finished blocks: the last
// block to finish writes the frame's row tables.
// (horizon block hblk, slope k of the frame's nblocks vote blocks)
__device__ __forceinline__ void vote_block(const int32_t* __restrict__ smooth, int H, int dmax,
                                           unsigned long long* __restrict__ best, const int32_t* __restrict__ kg_tab,
                                           const RowsDev& cam, const RealModelDev* __restrict__ rm,
                                           const int32_t* __restrict__ est_pool, int gw, double* __restrict__ rows,
                                           int32_t* __restrict__ pool, int32_t* __restrict__ line, const int hblk,
                                           const int k, const unsigned long long nblocks)
{
    __shared__ bool s_last;
    __shared__ int32_t s_v[kVoteWarps][kVoteH];
    const int E = 16 * dmax + 1, Hp = ground_pitch(H);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int hb = hblk * kVoteH, hl = hb + lane;
    // offsets j = r - h with code (k j + 8) >> 4 in [16, E): up to j_hi some
    // horizon of the block has its row r < H, up to j_all every one has
    const int j_lo = (248 + k - 1) / k;
    const int j_top = (16 * E - 9) / k;
    const int j_hi = min(j_top, H - 1 - hb);
    const int j_all = min(j_top, H - kVoteH - hb);
    const int32_t* __restrict__ base = smooth + hl;
    int32_t votes[kVoteM];
#pragma unroll
    for (int m = 0; m < kVoteM; ++m) votes[m] = 0;
    int j0 = j_lo + 8 * w;
    for (; j0 + 7 <= j_all; j0 += 8 * kVoteWarps) {
        int32_t part[8][kVoteM];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int j = j0 + i;
            const int32_t* p = base + ((k * j + 8) >> 4) * Hp + j;
#pragma unroll
            for (int m = 0; m < kVoteM; ++m) part[i][m] = __ldg(p + 32 * m);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int m = 0; m < kVoteM; ++m) votes[m] += part[i][m];
    }
    for (; j0 <= j_hi; j0 += 8 * kVoteWarps) {
        int32_t part[8][kVoteM];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int j = j0 + i;
            const int32_t* p = base + ((k * j + 8) >> 4) * Hp + j;
#pragma unroll
            for (int m = 0; m < kVoteM; ++m)
                part[i][m] = (j <= j_hi && hl + 32 * m + j < H) ? __ldg(p + 32 * m) : 0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int m = 0; m < kVoteM; ++m) votes[m] += part[i][m];
    }
#pragma unroll
    for (int m = 0; m < kVoteM; ++m) s_v[w][lane + 32 * m] = votes[m];
    __syncthreads();
    if (w == 0) {
        unsigned long long key = 0ull;
#pragma unroll
        for (int m = 0; m < kVoteM; ++m) {
            const int h = hl + 32 * m;
            int32_t v = 0;
#pragma unroll
            for (int i = 0; i < kVoteWarps; ++i) v += s_v[i][lane + 32 * m];
            const unsigned long long km = h < H ? ((unsigned long long)(uint32_t)v << 32) |
                                                      ((unsigned long long)(256 - k) << 16) |
                                                      (unsigned long long)(65535 - h)
                                                : 0ull;
            key = km > key ? km : key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other > key ? other : key;
        }
        if (lane == 0) {
            atomicMax(best, key);
            // the winner is visible before this block counts as finished
            __threadfence();
            const unsigned long long done = atomicAdd(best + 1, 1ull);
            s_last = done + 1 == nblocks;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    write_ground_rows(atomicAdd(best, 0ull), H, dmax, kg_tab, cam, rm, est_pool, gw, rows, pool, line);
}

__global__ void __launch_bounds__(32 * kVoteWarps) vote_kernel(const int32_t* __restrict__ smooth, int H,
                                                               int dmax, unsigned long long* __restrict__ best,
                                                               const int32_t* __restrict__ kg_tab, RowsDev cam,
                                                               const RealModelDev* __restrict__ rm,
                                                               const int32_t* __restrict__ est_pool, int gw,
                                                               double* __restrict__ rows, int32_t* __restrict__ pool,
                                                               int32_t* __restrict__ line)
{
    vote_block(smooth, H, dmax, best, kg_tab, cam, rm, est_pool, gw, rows, pool, line, blockIdx.x, blockIdx.y + 1,
               (unsigned long long)gridDim.x * gridDim.y);
}

// Batch forms: blockIdx.x indexes a list of (frame, row block) or (frame,
// horizon block) items; each frame's arguments come from its table row.
__global__ void __launch_bounds__(256) vdisp_batch_kernel(const GroundArgs* __restrict__ args,
                                                          const int2* __restrict__ items)
{
    const int2 w = items[blockIdx.x];
    const GroundArgs& a = args[w.x];
    vdisp_rows(a.q, a.H, a.ncols, a.dmax, a.smooth, a.best, w.y);
}

__global__ void __launch_bounds__(32 * kVoteWarps) vote_batch_kernel(const GroundArgs* __restrict__ args,
                                                                     const int2* __restrict__ items)
{
    const int2 w = items[blockIdx.x];
    const GroundArgs& a = args[w.x];
    vote_block(a.smooth, a.H, a.dmax, a.best, a.kg_tab, a.cam, a.rm, a.est_pool, a.gw, a.rows, a.pool, a.line, w.y,
               blockIdx.y + 1, (unsigned long long)a.nvote);
}

}  // namespace

// work layout: the smoothed table, the vote's winner and counter (256 bytes),
// the line {k, h, votes} (256 bytes), the frame's row tables (RowsDev), its
// residual windows (max(16, H) windows of gw codes)
static size_t smooth_bytes(int H, int dmax)
{
    return (sizeof(int32_t) * ground_pitch(H) * (16 * (size_t)dmax + 1) + 255) / 256 * 256;
}

static size_t frame_rows_bytes(int H) { return (rows_arrays_bytes(H) + 255) / 256 * 256; }

size_t ground_work_bytes(int H, int dmax, int gw)
{
    return smooth_bytes(H, dmax) + 256 + 256 + frame_rows_bytes(H) +
           sizeof(int32_t) * (size_t)(H > 16 ? H : 16) * gw;
}

// Layout of the work block: smoothed v-disparity, best vote, own line, the
// frame's row tables, its residual windows.
RowsDev ground_frame_rows(const FrameGeom& g, int dmax, const RowsDev& cam, int est_gw, char* work)
{
    char* rows = work + smooth_bytes(g.H, dmax) + 256 + 256;
    RowsDev r;
    r.fg = reinterpret_cast<const double*>(rows);
    r.real_model = cam.real_model;
    r.gpool = reinterpret_cast<const int32_t*>(rows + frame_rows_bytes(g.H));
    r.gw = est_gw;
    r.gn = (g.H > 16 ? g.H : 16) * est_gw;
    return r;
}

cudaError_t prepare_ground_kernels()
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        // dmax 255: 32.8 KB
        e = cudaFuncSetAttribute(vdisp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ground_vdisp_smem(STIXELS_MAX_DMAX));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(vdisp_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ground_vdisp_smem(STIXELS_MAX_DMAX));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    return cudaSuccess;
}

int ground_row_blocks(int H) { return (H + kVdispRows - 1) / kVdispRows; }
int ground_horizon_blocks(int H) { return (H + kVoteH - 1) / kVoteH; }
size_t ground_vdisp_smem(int dmax) { return sizeof(int32_t) * kVdispRows * vdisp_pitch(16 * dmax + 1); }

bool ground_args(const int16_t* q, const FrameGeom& g, const ModelDev& m, const RowsDev& cam, const int32_t* est_pool,
                 int est_gw, char* work, int32_t* line, GroundArgs* a)
{
    if (!est_pool || est_gw != cam.gw) return false;
    const RowsDev fr = ground_frame_rows(g, m.dmax, cam, est_gw, work);
    a->q = q;
    a->H = g.H;
    a->ncols = g.ncols;
    a->dmax = m.dmax;
    a->smooth = (int32_t*)work;
    a->best = (unsigned long long*)(work + smooth_bytes(g.H, m.dmax));
    a->kg_tab = m.kg_tab;
    a->cam = cam;
    a->rm = cam.real_model;
    a->est_pool = est_pool;
    a->gw = est_gw;
    a->rows = const_cast<double*>(fr.fg);
    a->pool = const_cast<int32_t*>(fr.gpool);
    a->line = line ? line : (int32_t*)((char*)a->best + 256);
    a->nvote = ground_horizon_blocks(g.H) * 256;
    return true;
}

cudaError_t launch_ground(const int16_t* q, const FrameGeom& g, const ModelDev& m, RowsDev cam,
                          const int32_t* est_pool, int est_gw, char* work, RowsDev* frame_rows, int32_t* line,
                          cudaStream_t st)
{
    // cam is a copy: frame_rows may be the caller's camera rows themselves
    GroundArgs a;
    if (!ground_args(q, g, m, cam, est_pool, est_gw, work, line, &a)) return cudaErrorInvalidValue;
    *frame_rows = ground_frame_rows(g, m.dmax, cam, est_gw, work);
    cudaError_t e = prepare_ground_kernels();
    if (e != cudaSuccess) return e;
    vdisp_kernel<<<ground_row_blocks(g.H), 256, ground_vdisp_smem(m.dmax), st>>>(q, g.H, g.ncols, m.dmax, a.smooth,
                                                                                  a.best);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vote_kernel<<<dim3(ground_horizon_blocks(g.H), 256), 32 * kVoteWarps, 0, st>>>(
        a.smooth, g.H, m.dmax, a.best, m.kg_tab, cam, cam.real_model, est_pool, est_gw, a.rows, a.pool, a.line);
    return cudaGetLastError();
}

cudaError_t launch_ground_batch(const GroundArgs* d_args, const int2* d_row_items, int nrow_items,
                                const int2* d_vote_items, int nvote_items, size_t vdisp_smem, cudaStream_t st)
{
    if (nrow_items <= 0 || nvote_items <= 0) return cudaSuccess;
    cudaError_t e = prepare_ground_kernels();
    if (e != cudaSuccess) return e;
    vdisp_batch_kernel<<<nrow_items, 256, vdisp_smem, st>>>(d_args, d_row_items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vote_batch_kernel<<<dim3(nvote_items, 256), 32 * kVoteWarps, 0, st>>>(d_args, d_vote_items);
    return cudaGetLastError();
}

}  // namespace stx
