// batch.cu -- batched mode: a fixed set of frames (each with its own camera
// handle and size) processed by one graph-captured launch sequence, with a
// persistent DP kernel over a longest-first column work list, and an autotuner
// for the DP launch shape.  The table planning here is shared with the server.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace stx {

namespace {
size_t up256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

namespace {
size_t ground_bytes(const FrameGeom& g, const HandleView& v)
{
    return v.ground_estimate ? up256(ground_work_bytes(g.H, v.model.dmax, v.est_gw)) : 0;
}
}  // namespace

size_t frame_work_bytes(const FrameGeom& g, const HandleView& v)
{
    const size_t C = (size_t)g.ncols, P = (size_t)g.P, F = (size_t)v.model.dmax + 1;
    return up256(sizeof(int16_t) * C * g.H) + 3 * up256(sizeof(int32_t) * C * P) + up256(sizeof(int32_t) * C * F * P) +
           ground_bytes(g, v) + (v.global_map ? up256(map_scratch_bytes(g.H, g.ncols, (int)F)) : 0);
}

void frame_work_carve(FrameJob* job, char* base)
{
    const FrameGeom& g = job->g;
    const size_t C = (size_t)g.ncols, P = (size_t)g.P, F = (size_t)job->view.model.dmax + 1;
    size_t off = 0;
    job->q = (int16_t*)(base + off);  off += up256(sizeof(int16_t) * C * g.H);
    job->pd = (int32_t*)(base + off); off += up256(sizeof(int32_t) * C * P);
    job->pg = (int32_t*)(base + off); off += up256(sizeof(int32_t) * C * P);
    job->ps = (int32_t*)(base + off); off += up256(sizeof(int32_t) * C * P);
    job->po = (int32_t*)(base + off); off += up256(sizeof(int32_t) * C * F * P);
    job->ground_work = job->view.ground_estimate ? base + off : nullptr;
    off += ground_bytes(g, job->view);
    job->map_scratch = job->view.global_map ? base + off : nullptr;
}

void plan_tables(const std::vector<FrameJob>& jobs, BatchTables* t)
{
    const int n = (int)jobs.size();
    std::vector<ReduceArgs> ra(n);
    std::vector<LutArgs> la(n);
    std::vector<DpArgs> da(n);
    std::vector<int2> lut_items, dp_items, map_items, ground_rows, ground_votes;
    std::vector<GroundArgs> ga(n);
    std::vector<MapScratch> ms(n, MapScratch{nullptr, nullptr, nullptr});
    std::vector<std::vector<int4>> group_tiles;
    t->groups.clear();
    t->maxH = t->max_groups = 0;
    t->lut_smem = 0;
    t->map_smem = 0;
    t->std_trans = true;
    t->ground_smem = 0;
    t->ground_ok = true;
    t->jobs = jobs;
    for (int i = 0; i < n; ++i) {
        const FrameJob& f = jobs[i];
        const ModelDev& m = f.view.model;
        // a frame with its ground estimated reads the row tables its ground
        // kernels write into its work block
        const RowsDev rows = f.view.ground_estimate
                                 ? ground_frame_rows(f.g, m.dmax, f.view.rows, f.view.est_gw, f.ground_work)
                                 : f.view.rows;
        ra[i].disp = f.in;
        ra[i].H = f.g.H; ra[i].W = f.g.W; ra[i].ncols = f.g.ncols; ra[i].dmax = m.dmax;
        ra[i].q = f.q;
        la[i].q = f.q;
        la[i].H = f.g.H; la[i].P = f.g.P; la[i].F = m.dmax + 1; la[i].m = m; la[i].rows = rows;
        la[i].pd = f.pd; la[i].pg = f.pg; la[i].ps = f.ps; la[i].po = f.po;
        la[i].range_only = 1;
        la[i].rows_per_cta = lut_rows_per_cta(m, 1);
        dp_frame_args(f.pd, f.pg, f.ps, f.po, f.g, m, rows, f.view.rp, f.view.pixel_floor, f.out, f.view.err, &da[i]);
        if (f.g.ncols == 0) continue;
        if (f.view.ground_estimate) {
            // its v-disparity and vote launches are shared with the batch's
            // other estimating frames
            if (ground_args(f.q, f.g, m, f.view.rows, f.view.est_pool, f.view.est_gw, f.ground_work, nullptr, &ga[i])) {
                t->ground_smem = std::max(t->ground_smem, ground_vdisp_smem(m.dmax));
                for (int rb = 0; rb < ground_row_blocks(f.g.H); ++rb) ground_rows.push_back(make_int2(i, rb));
                for (int hb = 0; hb < ground_horizon_blocks(f.g.H); ++hb) ground_votes.push_back(make_int2(i, hb));
            } else {
                t->ground_ok = false;
            }
        }
        t->max_groups = std::max(t->max_groups, lut_row_groups(m.dmax + 1, la[i].rows_per_cta));
        t->lut_smem = std::max(t->lut_smem, lut_shared_bytes(f.g.H, m));
        for (int c = 0; c < f.g.ncols; ++c) lut_items.push_back(make_int2(i, c));
        if (f.view.global_map) {
            // the global MAP: one launch over every such frame's columns,
            // after the persistent DP
            t->map_smem = std::max(t->map_smem, map_smem_bytes(f.g.H, m.dmax + 1));
            ms[i] = map_scratch_carve(f.map_scratch, f.g.H, f.g.ncols, m.dmax + 1);
            for (int c = 0; c < f.g.ncols; ++c) map_items.push_back(make_int2(i, c));
        } else {
            t->maxH = std::max(t->maxH, f.g.H);
            t->std_trans = t->std_trans && m.trans[1][1] >= kBig && m.trans[1][2] >= kBig && m.trans[2][2] >= kBig;
            for (int c = 0; c < f.g.ncols; ++c) dp_items.push_back(make_int2(i, c));
        }
        int gi = -1;
        for (size_t k = 0; k < t->groups.size(); ++k)
            if (t->groups[k].s == f.g.s && t->groups[k].mode == f.view.reduce_mode) gi = (int)k;
        if (gi < 0) {
            t->groups.push_back(ReduceGroup{f.g.s, f.view.reduce_mode, 0, 0});
            group_tiles.emplace_back();
            gi = (int)t->groups.size() - 1;
        }
        for (int c0 = 0; c0 < f.g.ncols; c0 += 32)
            for (int r0 = 0; r0 < f.g.H; r0 += 16) group_tiles[gi].push_back(make_int4(i, c0, r0, 0));
    }
    // DP work list: longest columns first (work grows as H^2), stable otherwise
    std::stable_sort(dp_items.begin(), dp_items.end(),
                     [&](const int2& x, const int2& y) { return jobs[x.x].g.H > jobs[y.x].g.H; });
    std::stable_sort(map_items.begin(), map_items.end(),
                     [&](const int2& x, const int2& y) { return jobs[x.x].g.H > jobs[y.x].g.H; });
    t->nitems = (int)dp_items.size();
    t->nlut = (int)lut_items.size();
    t->nmap = (int)map_items.size();
    t->ngr = (int)ground_rows.size();
    t->ngv = (int)ground_votes.size();

    size_t o = 0;
    t->o_red = o; o += up256(sizeof(ReduceArgs) * n);
    t->o_lut = o; o += up256(sizeof(LutArgs) * n);
    t->o_dp = o;  o += up256(sizeof(DpArgs) * n);
    t->o_li = o;  o += up256(sizeof(int2) * lut_items.size());
    t->o_di = o;  o += up256(sizeof(int2) * dp_items.size());
    t->o_cnt = o; o += 256;
    t->o_ms = o;  o += up256(sizeof(MapScratch) * n);
    t->o_mi = o;  o += up256(sizeof(int2) * map_items.size());
    t->o_ga = o;  o += up256(sizeof(GroundArgs) * n);
    t->o_gr = o;  o += up256(sizeof(int2) * ground_rows.size());
    t->o_gv = o;  o += up256(sizeof(int2) * ground_votes.size());
    for (size_t k = 0; k < t->groups.size(); ++k) {
        t->groups[k].tiles_off = o;
        t->groups[k].ntiles = (int)group_tiles[k].size();
        o += up256(sizeof(int4) * group_tiles[k].size());
    }
    t->host.assign(o, 0);
    char* h = t->host.data();
    memcpy(h + t->o_red, ra.data(), sizeof(ReduceArgs) * n);
    memcpy(h + t->o_lut, la.data(), sizeof(LutArgs) * n);
    memcpy(h + t->o_dp, da.data(), sizeof(DpArgs) * n);
    if (!lut_items.empty()) memcpy(h + t->o_li, lut_items.data(), sizeof(int2) * lut_items.size());
    if (!dp_items.empty()) memcpy(h + t->o_di, dp_items.data(), sizeof(int2) * dp_items.size());
    memcpy(h + t->o_ms, ms.data(), sizeof(MapScratch) * n);
    if (!map_items.empty()) memcpy(h + t->o_mi, map_items.data(), sizeof(int2) * map_items.size());
    memcpy(h + t->o_ga, ga.data(), sizeof(GroundArgs) * n);
    if (!ground_rows.empty()) memcpy(h + t->o_gr, ground_rows.data(), sizeof(int2) * ground_rows.size());
    if (!ground_votes.empty()) memcpy(h + t->o_gv, ground_votes.data(), sizeof(int2) * ground_votes.size());
    for (size_t k = 0; k < t->groups.size(); ++k)
        memcpy(h + t->groups[k].tiles_off, group_tiles[k].data(), sizeof(int4) * group_tiles[k].size());
}

cudaError_t launch_frame_job(const FrameJob& f, cudaStream_t st)
{
    const ModelDev& m = f.view.model;
    if (f.g.H <= 0 || f.g.ncols <= 0) return cudaSuccess;
    cudaError_t e = launch_reduce(f.in, f.g, m.dmax, f.view.reduce_mode, f.q, st);
    RowsDev r = f.view.rows;
    if (e == cudaSuccess && f.view.ground_estimate)
        e = launch_ground(f.q, f.g, m, r, f.view.est_pool, f.view.est_gw, f.ground_work, &r, nullptr, st);
    if (e == cudaSuccess) e = launch_luts(f.q, f.g, m, r, f.pd, f.pg, f.ps, f.po, st, 1);
    if (e == cudaSuccess)
        e = f.view.global_map ? launch_dp_map(f.pd, f.pg, f.ps, f.po, f.g, m, r, f.view.rp, f.view.pixel_floor, f.out,
                                              f.view.err, f.map_scratch, st)
                              : launch_dp(f.pd, f.pg, f.ps, f.po, f.g, m, r, f.view.rp, f.view.pixel_floor, f.out,
                                          f.view.err, st);
    return e;
}

cudaError_t enqueue_tables(const BatchTables& t, char* d_tab, int dp_warps, int dp_ctas_per_sm, cudaStream_t st)
{
    int* counter = (int*)(d_tab + t.o_cnt);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    for (const ReduceGroup& gr : t.groups) {
        if (e != cudaSuccess) return e;
        e = launch_reduce_batch((const ReduceArgs*)(d_tab + t.o_red), (const int4*)(d_tab + gr.tiles_off), gr.ntiles,
                                gr.s, gr.mode, st);
    }
    // frames that estimate their ground line: one v-disparity and one vote
    // launch over all of them write each frame's row tables, which its LUT
    // and DP arguments already point to
    if (e == cudaSuccess && !t.ground_ok) e = cudaErrorInvalidValue;
    if (e == cudaSuccess && t.ngr > 0)
        e = launch_ground_batch((const GroundArgs*)(d_tab + t.o_ga), (const int2*)(d_tab + t.o_gr), t.ngr,
                                (const int2*)(d_tab + t.o_gv), t.ngv, t.ground_smem, st);
    if (e == cudaSuccess)
        e = launch_luts_batch((const LutArgs*)(d_tab + t.o_lut), (const int2*)(d_tab + t.o_li), t.nlut, t.max_groups,
                              t.lut_smem, st);
    if (e == cudaSuccess && t.nitems > 0) {
        const int grid = std::max(1, std::min(t.nitems, sm_count() * dp_ctas_per_sm));
        e = launch_dp_batch((const DpArgs*)(d_tab + t.o_dp), (const int2*)(d_tab + t.o_di), t.nitems, counter, t.maxH,
                            dp_warps, dp_ctas_per_sm, t.std_trans, grid, st);
    }
    // frames solved by the global MAP: one launch over all their columns
    if (e == cudaSuccess && t.nmap > 0)
        e = launch_dp_map_batch((const DpArgs*)(d_tab + t.o_dp), (const MapScratch*)(d_tab + t.o_ms),
                                (const int2*)(d_tab + t.o_mi), t.nmap, t.map_smem, st);
    return e;
}

}  // namespace stx

using namespace stx;

namespace {

size_t up256b(size_t x) { return (x + 255) / 256 * 256; }

struct FramePlan {
    FrameJob job;
    size_t in_off, work_off, st_off, cnt_off, cost_off, fix_off;
};

}  // namespace

struct stixels_batch_s {
    int device = 0;
    std::vector<FramePlan> frames;
    BatchTables tables;
    void* d_mem = nullptr;                 // inputs, intermediates, outputs
    void* d_tab = nullptr;                 // argument tables and work lists
    size_t mem_bytes = 0;
    stixels_batch_config_t cfg{8, 2};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int capture(stixels_batch_t b)
{
    cudaError_t pe = prepare_dp_kernels();
    if (pe == cudaSuccess) pe = prepare_ground_kernels();
    if (pe == cudaSuccess) pe = prepare_map_kernel();
    if (pe != cudaSuccess) return status_from_cuda(pe);
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return status_from_cuda(e);
    cudaError_t e2 = enqueue_tables(b->tables, (char*)b->d_tab, b->cfg.dp_warps, b->cfg.dp_ctas_per_sm, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (e2 != cudaSuccess) return status_from_cuda(e2);
    if (e != cudaSuccess) return status_from_cuda(e);
    return status_from_cuda(cudaGraphInstantiate(&b->exec, b->graph, 0));
}

bool config_ok(const stixels_batch_config_t& c)
{
    return (c.dp_warps == 8 || c.dp_warps == 16) && c.dp_ctas_per_sm >= 1 && c.dp_ctas_per_sm <= 4 &&
           c.dp_warps * 32 * c.dp_ctas_per_sm <= 2048;
}

std::string batch_signature(stixels_batch_t b)
{
    std::vector<std::string> parts;
    for (const FramePlan& f : b->frames) {
        char buf[96];
        snprintf(buf, sizeof(buf), "%dx%d/s%d/d%d%s%s", f.job.g.W, f.job.g.H, f.job.g.s, f.job.view.model.dmax,
                 f.job.view.ground_estimate ? "/e" : "", f.job.view.global_map ? "/m" : "");
        parts.push_back(buf);
    }
    std::sort(parts.begin(), parts.end());
    std::string sig;
    for (size_t i = 0; i < parts.size();) {               // run-length: "count*shape,"
        size_t j = i;
        while (j < parts.size() && parts[j] == parts[i]) ++j;
        sig += std::to_string(j - i) + "*" + parts[i] + ",";
        i = j;
    }
    return sig;
}

}  // namespace

extern "C" {

int stixels_batch_create(const stixels_frame_desc_t* frames, int nframes, stixels_batch_t* out)
{
    if (!frames || nframes < 1 || !out) return STIXELS_E_INVALID_ARG;
    *out = nullptr;
    stixels_batch_s* b = new (std::nothrow) stixels_batch_s();
    if (!b) return STIXELS_E_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return STIXELS_E_CUDA; }
    // plan every frame and the memory layout
    size_t off = 0;
    for (int i = 0; i < nframes; ++i) {
        const stixels_frame_desc_t& d = frames[i];
        if (!d.camera || d.H < 1 || d.H > STIXELS_MAX_HEIGHT || d.W < 1 || d.W > (1 << 24)) {
            delete b;
            return STIXELS_E_INVALID_ARG;
        }
        FramePlan f;
        int rc = handle_prepare(d.camera, d.H, &f.job.view);
        if (rc != STIXELS_OK) { delete b; return rc; }
        if (f.job.view.device != b->device) { delete b; return STIXELS_E_INVALID_ARG; }
        FrameGeom& g = f.job.g;
        g.H = d.H; g.W = d.W; g.s = f.job.view.stixel_width; g.ncols = d.W / g.s; g.P = lut_pitch(d.H);
        if ((f.job.view.ground_estimate && !ground_size_ok(g)) ||
            (f.job.view.global_map && !map_fits(g.H, f.job.view.model.dmax + 1))) {
            delete b;
            return STIXELS_E_INVALID_ARG;
        }
        const size_t C = (size_t)g.ncols;
        f.in_off = off;   off += up256b(sizeof(float) * (size_t)d.H * d.W);
        f.work_off = off; off += frame_work_bytes(g, f.job.view);
        f.st_off = off;   off += up256b(sizeof(stixel_t) * C * f.job.view.capacity);
        f.cnt_off = off;  off += up256b(sizeof(int32_t) * C);
        f.cost_off = off; off += up256b(sizeof(float) * C);
        f.fix_off = off;  off += up256b(sizeof(int32_t) * C);
        b->frames.push_back(f);
    }
    b->mem_bytes = std::max<size_t>(off, 256);
    cudaError_t e = cudaMalloc(&b->d_mem, b->mem_bytes);
    if (e != cudaSuccess) { stixels_batch_destroy(b); return status_from_cuda(e); }
    char* mem = (char*)b->d_mem;
    std::vector<FrameJob> jobs;
    for (FramePlan& f : b->frames) {
        f.job.in = (const float*)(mem + f.in_off);
        frame_work_carve(&f.job, mem + f.work_off);
        f.job.out.stixels = (stixel_t*)(mem + f.st_off);
        f.job.out.counts = (int32_t*)(mem + f.cnt_off);
        f.job.out.column_cost = (float*)(mem + f.cost_off);
        f.job.out.column_cost_fixed = (int32_t*)(mem + f.fix_off);
        f.job.out.ncols = f.job.g.ncols;
        f.job.out.capacity = f.job.view.capacity;
        jobs.push_back(f.job);
    }
    plan_tables(jobs, &b->tables);
    e = cudaMalloc(&b->d_tab, b->tables.host.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tab, b->tables.host.data(), b->tables.host.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_mem, 0, b->mem_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { stixels_batch_destroy(b); return status_from_cuda(e); }
    int rc = capture(b);
    if (rc != STIXELS_OK) { stixels_batch_destroy(b); return rc; }
    *out = b;
    return STIXELS_OK;
}

int stixels_batch_input(stixels_batch_t b, int i, float** d_frame)
{
    if (!b || !d_frame || i < 0 || i >= (int)b->frames.size()) return STIXELS_E_INVALID_ARG;
    *d_frame = (float*)((char*)b->d_mem + b->frames[i].in_off);
    return STIXELS_OK;
}

int stixels_batch_output(stixels_batch_t b, int i, stixels_output_t* out)
{
    if (!b || !out || i < 0 || i >= (int)b->frames.size()) return STIXELS_E_INVALID_ARG;
    *out = b->frames[i].job.out;
    return STIXELS_OK;
}

int stixels_batch_set_input(stixels_batch_t b, int i, const float* src, void* stream)
{
    if (!b || !src || i < 0 || i >= (int)b->frames.size()) return STIXELS_E_INVALID_ARG;
    const FramePlan& f = b->frames[i];
    return status_from_cuda(cudaMemcpyAsync((char*)b->d_mem + f.in_off, src,
                                            sizeof(float) * (size_t)f.job.g.H * f.job.g.W, cudaMemcpyDefault,
                                            (cudaStream_t)stream));
}

int stixels_batch_get_output(stixels_batch_t b, int i, stixel_t* stixels, int32_t* counts, float* cost,
                             int32_t* cost_fixed, void* stream)
{
    if (!b || i < 0 || i >= (int)b->frames.size()) return STIXELS_E_INVALID_ARG;
    const stixels_output_t& o = b->frames[i].job.out;
    const size_t C = (size_t)o.ncols;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (stixels) e = cudaMemcpyAsync(stixels, o.stixels, sizeof(stixel_t) * C * o.capacity, cudaMemcpyDefault, st);
    if (e == cudaSuccess && counts) e = cudaMemcpyAsync(counts, o.counts, sizeof(int32_t) * C, cudaMemcpyDefault, st);
    if (e == cudaSuccess && cost) e = cudaMemcpyAsync(cost, o.column_cost, sizeof(float) * C, cudaMemcpyDefault, st);
    if (e == cudaSuccess && cost_fixed)
        e = cudaMemcpyAsync(cost_fixed, o.column_cost_fixed, sizeof(int32_t) * C, cudaMemcpyDefault, st);
    return status_from_cuda(e);
}

int stixels_batch_launch(stixels_batch_t b, void* stream)
{
    if (!b || !b->exec) return STIXELS_E_INVALID_ARG;
    return status_from_cuda(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int stixels_batch_set_config(stixels_batch_t b, const stixels_batch_config_t* cfg)
{
    if (!b || !cfg || !config_ok(*cfg)) return STIXELS_E_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return status_from_cuda(e);
    b->cfg = *cfg;
    return capture(b);
}

int stixels_batch_get_config(stixels_batch_t b, stixels_batch_config_t* cfg)
{
    if (!b || !cfg) return STIXELS_E_INVALID_ARG;
    *cfg = b->cfg;
    return STIXELS_OK;
}

int stixels_batch_tune(stixels_batch_t b, void* stream, const char* cache_path, stixels_batch_config_t* chosen)
{
    if (!b) return STIXELS_E_INVALID_ARG;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) return STIXELS_E_CUDA;
    const std::string key = std::string(prop.name) + "|" + batch_signature(b);
    // cached result?
    if (cache_path) {
        FILE* fh = fopen(cache_path, "r");
        if (fh) {
            char line[4096];
            stixels_batch_config_t hit{0, 0};
            while (fgets(line, sizeof(line), fh)) {
                const size_t len = strlen(line);
                if (len > key.size() && strncmp(line, key.c_str(), key.size()) == 0 && line[key.size()] == '\t') {
                    int w = 0, c = 0;
                    if (sscanf(line + key.size() + 1, "%d %d", &w, &c) == 2) hit = stixels_batch_config_t{w, c};
                }
            }
            fclose(fh);
            if (config_ok(hit)) {
                int rc = stixels_batch_set_config(b, &hit);
                if (rc == STIXELS_OK && chosen) *chosen = hit;
                return rc;
            }
        }
    }
    const stixels_batch_config_t cands[] = {{8, 2}, {16, 1}, {8, 1}, {8, 3}};
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return STIXELS_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return STIXELS_E_CUDA; }
    float best_ms = 0.0f;
    stixels_batch_config_t best = b->cfg;
    int rc = STIXELS_OK;
    for (const stixels_batch_config_t& c : cands) {
        rc = stixels_batch_set_config(b, &c);
        if (rc != STIXELS_OK) break;
        cudaError_t e = cudaGraphLaunch(b->exec, st);                 // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { rc = status_from_cuda(e); break; }
        if (best_ms == 0.0f || ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != STIXELS_OK) return rc;
    rc = stixels_batch_set_config(b, &best);
    if (rc != STIXELS_OK) return rc;
    if (chosen) *chosen = best;
    if (cache_path) {
        FILE* fh = fopen(cache_path, "a");
        if (fh) {
            fprintf(fh, "%s\t%d %d %.4f\n", key.c_str(), best.dp_warps, best.dp_ctas_per_sm, best_ms / 3.0f);
            fclose(fh);
        }
    }
    return STIXELS_OK;
}

int stixels_batch_destroy(stixels_batch_t b)
{
    if (!b) return STIXELS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_mem);
    cudaFree(b->d_tab);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
    return STIXELS_OK;
}

}  // extern "C"
