// batch.cu -- batched mode: a fixed set of frames (each with its own camera
// handle and size) processed by one graph-captured launch sequence, with a
// persistent DP kernel over a longest-first column work list, and an autotuner
// for the DP launch shape.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace stx;

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct FramePlan {
    stixels_t cam;
    HandleView view;
    FrameGeom g;
    size_t in_off, q_off, pd_off, pg_off, ps_off, po_off;
    size_t st_off, cnt_off, cost_off, fix_off;
};

struct ReduceGroup {            // frames sharing stixel width and reduction mode
    int s, mode;
    size_t tiles_off;           // offset of its int4 tiles in the table block
    int ntiles;
};

}  // namespace

struct stixels_batch_s {
    int device = 0;
    std::vector<FramePlan> frames;
    std::vector<ReduceGroup> groups;
    void* d_mem = nullptr;                 // inputs, intermediates, outputs
    void* d_tab = nullptr;                 // argument tables and work lists
    size_t mem_bytes = 0, tab_bytes = 0;
    ReduceArgs* d_reduce = nullptr;
    LutArgs* d_lut = nullptr;
    DpArgs* d_dp = nullptr;
    int2* d_lut_items = nullptr;
    int2* d_dp_items = nullptr;
    int* d_counter = nullptr;
    int nitems = 0, max_groups = 0, maxH = 0;
    size_t lut_smem = 0;
    bool std_trans = true;
    stixels_batch_config_t cfg{8, 2};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int status_of(cudaError_t e) { return status_from_cuda(e); }

cudaError_t enqueue(stixels_batch_t b, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
    for (const ReduceGroup& gr : b->groups) {
        if (e != cudaSuccess) return e;
        e = launch_reduce_batch(b->d_reduce, reinterpret_cast<const int4*>((char*)b->d_tab + gr.tiles_off), gr.ntiles,
                                gr.s, gr.mode, st);
    }
    if (e == cudaSuccess)
        e = launch_luts_batch(b->d_lut, b->d_lut_items, b->nitems, b->max_groups, b->lut_smem, st);
    if (e == cudaSuccess) {
        const int grid = std::max(1, std::min(b->nitems, sm_count() * b->cfg.dp_ctas_per_sm));
        e = launch_dp_batch(b->d_dp, b->d_dp_items, b->nitems, b->d_counter, b->maxH, b->cfg.dp_warps, b->std_trans,
                            grid, st);
    }
    return e;
}

int capture(stixels_batch_t b)
{
    cudaError_t pe = prepare_dp_kernels();
    if (pe != cudaSuccess) return status_of(pe);
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return status_of(e);
    cudaError_t e2 = enqueue(b, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (e2 != cudaSuccess) return status_of(e2);
    if (e != cudaSuccess) return status_of(e);
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    return status_of(e);
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
        snprintf(buf, sizeof(buf), "%dx%d/s%d/d%d", f.g.W, f.g.H, f.g.s, f.view.model.dmax);
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
        FramePlan f;
        f.cam = d.camera;
        if (!d.camera || d.H < 1 || d.H > STIXELS_MAX_HEIGHT || d.W < 1 || d.W > (1 << 24)) {
            delete b;
            return STIXELS_E_INVALID_ARG;
        }
        int rc = handle_prepare(d.camera, d.H, &f.view);
        if (rc != STIXELS_OK) { delete b; return rc; }
        if (f.view.device != b->device) { delete b; return STIXELS_E_INVALID_ARG; }
        f.g.H = d.H; f.g.W = d.W; f.g.s = f.view.stixel_width; f.g.ncols = d.W / f.g.s; f.g.P = lut_pitch(d.H);
        const size_t C = (size_t)f.g.ncols, P = (size_t)f.g.P, F = (size_t)f.view.model.dmax + 1;
        f.in_off = off;   off += up256(sizeof(float) * (size_t)d.H * d.W);
        f.q_off = off;    off += up256(sizeof(int16_t) * C * d.H);
        f.pd_off = off;   off += up256(sizeof(int32_t) * C * P);
        f.pg_off = off;   off += up256(sizeof(int32_t) * C * P);
        f.ps_off = off;   off += up256(sizeof(int32_t) * C * P);
        f.po_off = off;   off += up256(sizeof(int32_t) * C * F * P);
        f.st_off = off;   off += up256(sizeof(stixel_t) * C * f.view.capacity);
        f.cnt_off = off;  off += up256(sizeof(int32_t) * C);
        f.cost_off = off; off += up256(sizeof(float) * C);
        f.fix_off = off;  off += up256(sizeof(int32_t) * C);
        b->frames.push_back(f);
    }
    b->mem_bytes = std::max<size_t>(off, 256);
    cudaError_t e = cudaMalloc(&b->d_mem, b->mem_bytes);
    if (e != cudaSuccess) { stixels_batch_destroy(b); return status_of(e); }
    char* mem = (char*)b->d_mem;

    // host-side tables
    const int n = nframes;
    std::vector<ReduceArgs> ra(n);
    std::vector<LutArgs> la(n);
    std::vector<DpArgs> da(n);
    std::vector<int2> lut_items, dp_items;
    std::vector<std::vector<int4>> group_tiles;
    for (int i = 0; i < n; ++i) {
        FramePlan& f = b->frames[i];
        const ModelDev& m = f.view.model;
        ra[i].disp = (const float*)(mem + f.in_off);
        ra[i].H = f.g.H; ra[i].W = f.g.W; ra[i].ncols = f.g.ncols; ra[i].dmax = m.dmax;
        ra[i].q = (int16_t*)(mem + f.q_off);
        la[i].q = (const int16_t*)(mem + f.q_off);
        la[i].H = f.g.H; la[i].P = f.g.P; la[i].F = m.dmax + 1; la[i].m = m; la[i].rows = f.view.rows;
        la[i].pd = (int32_t*)(mem + f.pd_off); la[i].pg = (int32_t*)(mem + f.pg_off);
        la[i].ps = (int32_t*)(mem + f.ps_off); la[i].po = (int32_t*)(mem + f.po_off);
        stixels_output_t o;
        o.stixels = (stixel_t*)(mem + f.st_off); o.counts = (int32_t*)(mem + f.cnt_off);
        o.column_cost = (float*)(mem + f.cost_off); o.column_cost_fixed = (int32_t*)(mem + f.fix_off);
        o.ncols = f.g.ncols; o.capacity = f.view.capacity;
        dp_frame_args(la[i].pd, la[i].pg, la[i].ps, la[i].po, f.g, m, f.view.rows, o, f.view.err, &da[i]);
        b->maxH = std::max(b->maxH, f.g.H);
        b->max_groups = std::max(b->max_groups, lut_row_groups(m.dmax + 1));
        b->lut_smem = std::max(b->lut_smem, lut_shared_bytes(f.g.H, m));
        b->std_trans = b->std_trans && m.trans[1][1] >= kBig && m.trans[1][2] >= kBig && m.trans[2][2] >= kBig;
        for (int c = 0; c < f.g.ncols; ++c) {
            lut_items.push_back(make_int2(i, c));
            dp_items.push_back(make_int2(i, c));
        }
        // reduction tiles, grouped by (stixel width, mode)
        int gi = -1;
        for (size_t k = 0; k < b->groups.size(); ++k)
            if (b->groups[k].s == f.g.s && b->groups[k].mode == f.view.reduce_mode) gi = (int)k;
        if (gi < 0) {
            b->groups.push_back(ReduceGroup{f.g.s, f.view.reduce_mode, 0, 0});
            group_tiles.emplace_back();
            gi = (int)b->groups.size() - 1;
        }
        for (int c0 = 0; c0 < f.g.ncols; c0 += 32)
            for (int r0 = 0; r0 < f.g.H; r0 += 16) group_tiles[gi].push_back(make_int4(i, c0, r0, 0));
    }
    // DP work list: longest columns first (work grows as H^2), stable otherwise
    std::stable_sort(dp_items.begin(), dp_items.end(), [&](const int2& x, const int2& y) {
        return b->frames[x.x].g.H > b->frames[y.x].g.H;
    });
    b->nitems = (int)dp_items.size();

    // device tables in one block
    size_t t = 0;
    const size_t o_red = t;  t += up256(sizeof(ReduceArgs) * n);
    const size_t o_lut = t;  t += up256(sizeof(LutArgs) * n);
    const size_t o_dp = t;   t += up256(sizeof(DpArgs) * n);
    const size_t o_li = t;   t += up256(sizeof(int2) * lut_items.size());
    const size_t o_di = t;   t += up256(sizeof(int2) * dp_items.size());
    const size_t o_cnt = t;  t += 256;
    for (size_t k = 0; k < b->groups.size(); ++k) {
        b->groups[k].tiles_off = t;
        b->groups[k].ntiles = (int)group_tiles[k].size();
        t += up256(sizeof(int4) * group_tiles[k].size());
    }
    b->tab_bytes = t;
    std::vector<char> host(t, 0);
    memcpy(host.data() + o_red, ra.data(), sizeof(ReduceArgs) * n);
    memcpy(host.data() + o_lut, la.data(), sizeof(LutArgs) * n);
    memcpy(host.data() + o_dp, da.data(), sizeof(DpArgs) * n);
    memcpy(host.data() + o_li, lut_items.data(), sizeof(int2) * lut_items.size());
    memcpy(host.data() + o_di, dp_items.data(), sizeof(int2) * dp_items.size());
    for (size_t k = 0; k < b->groups.size(); ++k)
        memcpy(host.data() + b->groups[k].tiles_off, group_tiles[k].data(), sizeof(int4) * group_tiles[k].size());
    e = cudaMalloc(&b->d_tab, t);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tab, host.data(), t, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_mem, 0, b->mem_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { stixels_batch_destroy(b); return status_of(e); }
    char* tab = (char*)b->d_tab;
    b->d_reduce = (ReduceArgs*)(tab + o_red);
    b->d_lut = (LutArgs*)(tab + o_lut);
    b->d_dp = (DpArgs*)(tab + o_dp);
    b->d_lut_items = (int2*)(tab + o_li);
    b->d_dp_items = (int2*)(tab + o_di);
    b->d_counter = (int*)(tab + o_cnt);
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
    const FramePlan& f = b->frames[i];
    char* mem = (char*)b->d_mem;
    out->stixels = (stixel_t*)(mem + f.st_off);
    out->counts = (int32_t*)(mem + f.cnt_off);
    out->column_cost = (float*)(mem + f.cost_off);
    out->column_cost_fixed = (int32_t*)(mem + f.fix_off);
    out->ncols = f.g.ncols;
    out->capacity = f.view.capacity;
    return STIXELS_OK;
}

int stixels_batch_set_input(stixels_batch_t b, int i, const float* src, void* stream)
{
    if (!b || !src || i < 0 || i >= (int)b->frames.size()) return STIXELS_E_INVALID_ARG;
    const FramePlan& f = b->frames[i];
    return status_of(cudaMemcpyAsync((char*)b->d_mem + f.in_off, src, sizeof(float) * (size_t)f.g.H * f.g.W,
                                     cudaMemcpyDefault, (cudaStream_t)stream));
}

int stixels_batch_get_output(stixels_batch_t b, int i, stixel_t* stixels, int32_t* counts, float* cost,
                             int32_t* cost_fixed, void* stream)
{
    if (!b || i < 0 || i >= (int)b->frames.size()) return STIXELS_E_INVALID_ARG;
    const FramePlan& f = b->frames[i];
    const char* mem = (const char*)b->d_mem;
    const size_t C = (size_t)f.g.ncols;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (stixels) e = cudaMemcpyAsync(stixels, mem + f.st_off, sizeof(stixel_t) * C * f.view.capacity, cudaMemcpyDefault, st);
    if (e == cudaSuccess && counts) e = cudaMemcpyAsync(counts, mem + f.cnt_off, sizeof(int32_t) * C, cudaMemcpyDefault, st);
    if (e == cudaSuccess && cost) e = cudaMemcpyAsync(cost, mem + f.cost_off, sizeof(float) * C, cudaMemcpyDefault, st);
    if (e == cudaSuccess && cost_fixed)
        e = cudaMemcpyAsync(cost_fixed, mem + f.fix_off, sizeof(int32_t) * C, cudaMemcpyDefault, st);
    return status_of(e);
}

int stixels_batch_launch(stixels_batch_t b, void* stream)
{
    if (!b || !b->exec) return STIXELS_E_INVALID_ARG;
    return status_of(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int stixels_batch_set_config(stixels_batch_t b, const stixels_batch_config_t* cfg)
{
    if (!b || !cfg || !config_ok(*cfg)) return STIXELS_E_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return status_of(e);
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
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return STIXELS_E_CUDA;
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
        if (e != cudaSuccess) { rc = status_of(e); break; }
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
