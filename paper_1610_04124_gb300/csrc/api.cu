// api.cu -- the C ABI of stixels.h: handles, workspace, per-frame pipeline.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "model.h"

using namespace stx;

namespace {

// Per-height row tables resident on the device.
struct RowsBuf {
    double* d = nullptr;    // the row tables of one height (RowsDev), then the rows' residual windows
    int H = 0, gw = 0;
};

struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Layout of one frame's intermediates inside a workspace.
struct FrameLayout {
    size_t q, pd, pg, ps, po, total;
};

FrameLayout frame_layout(int H, int ncols, int F)
{
    const int P = lut_pitch(H);
    FrameLayout L;
    size_t off = 0;
    L.q = off;  off = align_up(off + sizeof(int16_t) * (size_t)ncols * H, 256);
    L.pd = off; off = align_up(off + sizeof(int32_t) * (size_t)ncols * P, 256);
    L.pg = off; off = align_up(off + sizeof(int32_t) * (size_t)ncols * P, 256);
    L.ps = off; off = align_up(off + sizeof(int32_t) * (size_t)ncols * P, 256);
    L.po = off; off = align_up(off + sizeof(int32_t) * (size_t)ncols * F * P, 256);
    L.total = off;
    return L;
}

int cuda_status(cudaError_t e) { return stx::status_from_cuda(e); }

}  // namespace

struct stixels_s {
    int device = 0;
    HostModel hm;
    int32_t* d_tables = nullptr;       // k_obj | g_obj | g_sky | lut_cost | kg_tab | est_pool
    void* d_real = nullptr;            // RealModelDev, then its k_obj | inv_obj | rkg_tab
    RealParams rp;                     // the cost report's priors and constants (DP kernel arguments)
    const int32_t* est_pool = nullptr; // ground estimate: the residual windows of estimated lines (in d_tables)
    ModelDev md;
    std::map<int, RowsBuf> rows;       // per height
    Workspace ws;
    uint32_t* d_err = nullptr;
    uint32_t* h_err = nullptr;         // pinned copy of the error word (compute_host)
    cudaStream_t stream = nullptr;     // own stream for compute_host
    // device buffers for compute_host
    float* d_in = nullptr;
    size_t in_bytes = 0;
    void* d_out = nullptr;
    size_t out_bytes = 0;
};

namespace {

RowsDev rows_of(stixels_t h, const RowsBuf& rb)
{
    RowsDev r;
    r.fg = rb.d;
    r.real_model = static_cast<const RealModelDev*>(h->d_real);
    r.gpool = reinterpret_cast<const int32_t*>(reinterpret_cast<const char*>(rb.d) + rows_arrays_bytes(rb.H));
    r.gw = rb.gw;
    r.gn = rb.H * rb.gw;
    return r;
}

int ensure_rows(stixels_t h, int H, RowsDev* out)
{
    auto it = h->rows.find(H);
    if (it == h->rows.end()) {
        std::vector<char> block;
        RowsBuf rb;
        if (!build_rows(h->hm, H, &block, &rb.gw)) return STIXELS_E_INVALID_ARG;
        rb.H = H;
        cudaError_t e = cudaMalloc(&rb.d, block.size());
        if (e == cudaSuccess) e = cudaMemcpy(rb.d, block.data(), block.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(rb.d);
            return cuda_status(e);
        }
        it = h->rows.emplace(H, rb).first;
    }
    *out = rows_of(h, it->second);
    return STIXELS_OK;
}

int ensure_workspace(stixels_t h, size_t bytes)
{
    if (h->ws.bytes >= bytes) return STIXELS_OK;
    if (h->ws.base) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(h->ws.base);
        h->ws.base = nullptr;
        h->ws.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&h->ws.base, bytes);
    if (e != cudaSuccess) { h->ws.base = nullptr; return cuda_status(e); }
    h->ws.bytes = bytes;
    return STIXELS_OK;
}

int check_frame(stixels_t h, int H, int W)
{
    if (!h) return STIXELS_E_INVALID_ARG;
    if (H < 0 || W < 0 || H > STIXELS_MAX_HEIGHT) return STIXELS_E_INVALID_ARG;
    if (W > (1 << 24)) return STIXELS_E_INVALID_ARG;
    return STIXELS_OK;
}


FrameGeom geom(stixels_t h, int H, int W)
{
    FrameGeom g;
    g.H = H;
    g.W = W;
    g.s = h->hm.p.stixel_width;
    g.ncols = W / g.s;
    g.P = lut_pitch(H);
    return g;
}

int check_output(stixels_t h, const FrameGeom& g, const stixels_output_t* out)
{
    if (!out) return STIXELS_E_INVALID_ARG;
    if (out->ncols != g.ncols || out->capacity != h->hm.p.max_stixels_per_col) return STIXELS_E_INVALID_ARG;
    if (g.ncols > 0 && (!out->stixels || !out->counts)) return STIXELS_E_INVALID_ARG;
    return STIXELS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace stx {

namespace {
thread_local const char* t_last_cuda_error = "no error";
}

const char* t_last_cuda_error_string() { return t_last_cuda_error; }

int status_from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return STIXELS_OK;
    t_last_cuda_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STIXELS_E_OOM : STIXELS_E_CUDA;
}

// Read-only view of a handle for a frame of height H, without creating
// anything: fails with INVALID_ARG if the row tables for H do not exist yet.
int handle_view(stixels_t h, int H, HandleView* v)
{
    if (!h || !v) return STIXELS_E_INVALID_ARG;
    auto it = h->rows.find(H);
    if (it == h->rows.end()) return STIXELS_E_INVALID_ARG;
    v->device = h->device;
    v->model = h->md;
    v->rows = rows_of(h, it->second);
    v->rp = h->rp;
    v->pixel_floor = h->hm.pixel_floor;
    v->err = h->d_err;
    v->stixel_width = h->hm.p.stixel_width;
    v->reduce_mode = reduce_code(h->hm.p);
    v->ground_estimate = h->hm.p.ground_estimate;
    v->global_map = h->hm.p.global_map;
    v->est_pool = h->est_pool;
    v->est_gw = h->hm.est_gw;
    v->capacity = h->hm.p.max_stixels_per_col;
    return STIXELS_OK;
}

// As handle_view, creating the row tables for H first if needed (allocates).
int handle_prepare(stixels_t h, int H, HandleView* v)
{
    if (!h || H < 1 || H > STIXELS_MAX_HEIGHT) return STIXELS_E_INVALID_ARG;
    RowsDev r;
    int rc = ensure_rows(h, H, &r);
    if (rc) return rc;
    return handle_view(h, H, v);
}

}  // namespace stx

extern "C" {

int stixels_params_default(stixels_params_t* p)
{
    if (!p) return STIXELS_E_INVALID_ARG;
    default_params(p);
    return STIXELS_OK;
}

int stixels_create(const stixels_params_t* params, stixels_t* out_handle)
{
    if (!params || !out_handle) return STIXELS_E_INVALID_ARG;
    *out_handle = nullptr;
    stixels_s* h = new (std::nothrow) stixels_s();
    if (!h) return STIXELS_E_OOM;
    int rc = build_model(params, &h->hm);
    if (rc != STIXELS_OK) { delete h; return rc; }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return cuda_status(e); }
    const HostModel& m = h->hm;
    const size_t n_tab = m.k_obj.size() + m.g_obj.size() + m.g_sky.size() + m.lut_cost.size() + m.kg_tab.size() +
                         m.est_pool.size();
    e = cudaMalloc(&h->d_tables, sizeof(int32_t) * n_tab);
    if (e == cudaSuccess) {
        std::vector<int32_t> buf;
        buf.reserve(n_tab);
        buf.insert(buf.end(), m.k_obj.begin(), m.k_obj.end());
        buf.insert(buf.end(), m.g_obj.begin(), m.g_obj.end());
        buf.insert(buf.end(), m.g_sky.begin(), m.g_sky.end());
        buf.insert(buf.end(), m.lut_cost.begin(), m.lut_cost.end());
        buf.insert(buf.end(), m.kg_tab.begin(), m.kg_tab.end());
        buf.insert(buf.end(), m.est_pool.begin(), m.est_pool.end());
        e = cudaMemcpy(h->d_tables, buf.data(), sizeof(int32_t) * n_tab, cudaMemcpyHostToDevice);
    }
    // the model without the grid: the struct, then its per-f tables
    const size_t F = m.real.k_obj.size(), NK = m.real.rkg_tab.size();
    const size_t real_bytes = sizeof(RealModelDev) + sizeof(float) * (2 * F + NK);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_real, real_bytes);
    if (e == cudaSuccess) {
        std::vector<char> buf(real_bytes);
        RealModelDev rd;
        memset(&rd, 0, sizeof(rd));
        const RealModel& r = m.real;
        RealParams& rp = rd.rp;
        auto units = [](double x) {
            return std::isinf(x) ? kReportInf : (long long)llround(x * (double)kReportUnits);
        };
        for (int c = 0; c < 3; ++c) {
            rp.first[c] = units(r.first[c]);
            for (int q = 0; q < 3; ++q) rp.trans[c][q] = units(r.trans[c][q]);
        }
        rp.pen_grav = units(r.pen_grav);
        rp.pen_div = units(r.pen_div);
        rp.pen_ord = units(r.pen_ord);
        rp.c_out = r.c_out;
        rp.k_sky = r.k_sky;
        rp.inv_sky = r.inv_sky;
        h->rp = rp;
        rd.eps_g = r.eps_g;
        rd.eps_d = r.eps_d;
        rd.inv_ground = r.inv_ground;
        rd.dmax = m.dmax;
        // k_obj, inv_obj and rkg_tab follow the struct (the kernels address them from it)
        float* tk = reinterpret_cast<float*>((char*)h->d_real + sizeof(RealModelDev));
        rd.rkg_tab = NK ? tk + 2 * F : nullptr;
        memcpy(buf.data(), &rd, sizeof(rd));
        memcpy(buf.data() + sizeof(rd), r.k_obj.data(), sizeof(float) * F);
        memcpy(buf.data() + sizeof(rd) + sizeof(float) * F, r.inv_obj.data(), sizeof(float) * F);
        if (NK) memcpy(buf.data() + sizeof(rd) + sizeof(float) * 2 * F, r.rkg_tab.data(), sizeof(float) * NK);
        e = cudaMemcpy(h->d_real, buf.data(), real_bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        stixels_destroy(h);
        return cuda_status(e);
    }
    ModelDev& d = h->md;
    d.dmax = m.dmax;
    d.emax = m.emax;
    d.c_out = m.c_out;
    d.k_sky = m.k_sky;
    for (int c = 0; c < 3; ++c) {
        d.first[c] = m.first[c];
        for (int q = 0; q < 3; ++q) d.trans[c][q] = m.trans[c][q];
    }
    d.pen_grav = m.pen_grav;
    d.pen_div = m.pen_div;
    d.pen_ord = m.pen_ord;
    d.ord_off = m.ord_off;
    d.esat_obj = m.esat[0];
    d.esat_sky = m.esat[2];
    d.k_obj = h->d_tables;
    d.g_obj = d.k_obj + m.k_obj.size();
    d.g_sky = d.g_obj + m.g_obj.size();
    d.var_sigma = m.var_sigma ? 1 : 0;
    d.int_grid = m.p.pixel_grid;
    d.lut_cost = m.p.pixel_grid ? d.g_sky + m.g_sky.size() : nullptr;
    d.kg_tab = m.p.ground_estimate ? d.g_sky + m.g_sky.size() + m.lut_cost.size() : nullptr;
    h->est_pool = m.p.ground_estimate ? d.g_sky + m.g_sky.size() + m.lut_cost.size() + m.kg_tab.size() : nullptr;
    *out_handle = h;
    return STIXELS_OK;
}

int stixels_destroy(stixels_t h)
{
    if (!h) return STIXELS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto& kv : h->rows) cudaFree(kv.second.d);
    cudaFree(h->ws.base);
    cudaFree(h->d_tables);
    cudaFree(h->d_real);
    cudaFree(h->d_err);
    if (h->h_err) cudaFreeHost(h->h_err);
    cudaFree(h->d_in);
    cudaFree(h->d_out);
    if (h->stream) cudaStreamDestroy(h->stream);
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
    return STIXELS_OK;
}

int stixels_output_shape(stixels_t h, int H, int W, int* ncols, int* capacity)
{
    int rc = check_frame(h, H, W);
    if (rc) return rc;
    if (ncols) *ncols = W / h->hm.p.stixel_width;
    if (capacity) *capacity = h->hm.p.max_stixels_per_col;
    return STIXELS_OK;
}

int stixels_lut_pitch(int H) { return H < 0 ? 0 : lut_pitch(H); }

int stixels_reserve(stixels_t h, int H, int W)
{
    int rc = check_frame(h, H, W);
    if (rc) return rc;
    if (H == 0) return STIXELS_OK;
    RowsDev r;
    rc = ensure_rows(h, H, &r);
    if (rc) return rc;
    const FrameGeom g = geom(h, H, W);
    return ensure_workspace(h, frame_layout(H, g.ncols, h->hm.dmax + 1).total);
}

int stixels_reduce(stixels_t h, const float* d_disparity, int H, int W, void* stream, int16_t* d_q)
{
    int rc = check_frame(h, H, W);
    if (rc) return rc;
    const FrameGeom g = geom(h, H, W);
    if (g.H == 0 || g.ncols == 0) return STIXELS_OK;
    if (!d_disparity || !d_q) return STIXELS_E_INVALID_ARG;
    return cuda_status(launch_reduce(d_disparity, g, h->hm.dmax, reduce_code(h->hm.p), d_q, (cudaStream_t)stream));
}

int stixels_estimate_ground(stixels_t h, const int16_t* d_q, int H, int ncols, void* stream, int32_t* d_line)
{
    if (!h || H < 0 || H > STIXELS_MAX_HEIGHT || ncols < 0) return STIXELS_E_INVALID_ARG;
    if (H == 0 || ncols == 0) return STIXELS_OK;
    if (!d_q || !d_line || !h->md.kg_tab) return STIXELS_E_INVALID_ARG;
    FrameGeom g;
    g.H = H; g.W = ncols * h->hm.p.stixel_width; g.s = h->hm.p.stixel_width; g.ncols = ncols; g.P = lut_pitch(H);
    if (!ground_size_ok(g)) return STIXELS_E_INVALID_ARG;
    RowsDev r;
    int rc = ensure_rows(h, H, &r);
    if (rc) return rc;
    rc = ensure_workspace(h, ground_work_bytes(H, h->hm.dmax, h->hm.est_gw));
    if (rc) return rc;
    RowsDev fr;
    return cuda_status(launch_ground(d_q, g, h->md, r, h->est_pool, h->hm.est_gw, (char*)h->ws.base, &fr, d_line,
                                     (cudaStream_t)stream));
}

int stixels_build_luts(stixels_t h, const int16_t* d_q, int H, int ncols, void* stream, int32_t* d_pd,
                       int32_t* d_pg, int32_t* d_ps, int32_t* d_po)
{
    if (!h || H < 0 || H > STIXELS_MAX_HEIGHT || ncols < 0) return STIXELS_E_INVALID_ARG;
    if (H == 0 || ncols == 0) return STIXELS_OK;
    if (!d_q || !d_pd || !d_pg || !d_ps || !d_po) return STIXELS_E_INVALID_ARG;
    if (!aligned16(d_pd) || !aligned16(d_pg) || !aligned16(d_ps) || !aligned16(d_po)) return STIXELS_E_INVALID_ARG;
    RowsDev r;
    int rc = ensure_rows(h, H, &r);
    if (rc) return rc;
    FrameGeom g;
    g.H = H; g.W = ncols * h->hm.p.stixel_width; g.s = h->hm.p.stixel_width; g.ncols = ncols; g.P = lut_pitch(H);
    return cuda_status(launch_luts(d_q, g, h->md, r, d_pd, d_pg, d_ps, d_po, (cudaStream_t)stream));
}

int stixels_solve(stixels_t h, const int32_t* d_pd, const int32_t* d_pg, const int32_t* d_ps, const int32_t* d_po,
                  int H, int ncols, void* stream, const stixels_output_t* out)
{
    if (!h || H < 0 || H > STIXELS_MAX_HEIGHT || ncols < 0) return STIXELS_E_INVALID_ARG;
    FrameGeom g;
    g.H = H; g.W = ncols * h->hm.p.stixel_width; g.s = h->hm.p.stixel_width; g.ncols = ncols; g.P = lut_pitch(H);
    int rc = check_output(h, g, out);
    if (rc) return rc;
    if (H == 0 || ncols == 0) return STIXELS_OK;
    if (!d_pd || !d_pg || !d_ps || !d_po) return STIXELS_E_INVALID_ARG;
    RowsDev r;
    rc = ensure_rows(h, H, &r);
    if (rc) return rc;
    if (h->hm.p.global_map) {
        if (!map_fits(H, h->hm.dmax + 1)) return STIXELS_E_INVALID_ARG;
        rc = ensure_workspace(h, map_scratch_bytes(H, ncols, h->hm.dmax + 1));
        if (rc) return rc;
        return cuda_status(launch_dp_map(d_pd, d_pg, d_ps, d_po, g, h->md, r, h->rp, h->hm.pixel_floor, *out, h->d_err, h->ws.base,
                                         (cudaStream_t)stream));
    }
    return cuda_status(launch_dp(d_pd, d_pg, d_ps, d_po, g, h->md, r, h->rp, h->hm.pixel_floor, *out, h->d_err, (cudaStream_t)stream));
}

// The pipeline of stixels_compute, with the kernels' status flags ORed into
// `err` (device-addressable; the handle's error word for stixels_compute).
static int compute_frame(stixels_t h, const float* d_disparity, int H, int W, void* stream,
                         const stixels_output_t* out, uint32_t* err)
{
    int rc = check_frame(h, H, W);
    if (rc) return rc;
    const FrameGeom g = geom(h, H, W);
    rc = check_output(h, g, out);
    if (rc) return rc;
    if (g.H == 0 || g.ncols == 0) return STIXELS_OK;
    if (!d_disparity) return STIXELS_E_INVALID_ARG;
    RowsDev r;
    rc = ensure_rows(h, H, &r);
    if (rc) return rc;
    const bool est = h->hm.p.ground_estimate != 0;
    if (est && !ground_size_ok(g)) return STIXELS_E_INVALID_ARG;
    const FrameLayout L = frame_layout(H, g.ncols, h->hm.dmax + 1);
    const size_t gw = est ? (ground_work_bytes(H, h->hm.dmax, h->hm.est_gw) + 255) / 256 * 256 : 0;
    const bool gmap = h->hm.p.global_map != 0;
    if (gmap && !map_fits(H, h->hm.dmax + 1)) return STIXELS_E_INVALID_ARG;
    rc = ensure_workspace(h, L.total + gw + (gmap ? map_scratch_bytes(H, g.ncols, h->hm.dmax + 1) : 0));
    if (rc) return rc;
    char* ws = (char*)h->ws.base;
    int16_t* q = (int16_t*)(ws + L.q);
    int32_t* pd = (int32_t*)(ws + L.pd);
    int32_t* pg = (int32_t*)(ws + L.pg);
    int32_t* ps = (int32_t*)(ws + L.ps);
    int32_t* po = (int32_t*)(ws + L.po);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_reduce(d_disparity, g, h->hm.dmax, reduce_code(h->hm.p), q, st);
    if (e == cudaSuccess && est) e = launch_ground(q, g, h->md, r, h->est_pool, h->hm.est_gw, ws + L.total, &r, nullptr, st);
    if (e == cudaSuccess) e = launch_luts(q, g, h->md, r, pd, pg, ps, po, st, 1);
    if (e == cudaSuccess)
        e = gmap ? launch_dp_map(pd, pg, ps, po, g, h->md, r, h->rp, h->hm.pixel_floor, *out, err, ws + L.total + gw, st)
                 : launch_dp(pd, pg, ps, po, g, h->md, r, h->rp, h->hm.pixel_floor, *out, err, st);
    return cuda_status(e);
}

int stixels_compute(stixels_t h, const float* d_disparity, int H, int W, void* stream, const stixels_output_t* out)
{
    return compute_frame(h, d_disparity, H, W, stream, out, h ? h->d_err : nullptr);
}

int stixels_selftest_wait(stixels_t h, int polls, void* stream, uint32_t* flags)
{
    if (!h || !flags || polls < 1 || polls > (1 << 22)) return STIXELS_E_INVALID_ARG;
    const int rc = cuda_status(launch_wait_selftest(h->d_err, polls, (cudaStream_t)stream));
    if (rc) return rc;
    return stixels_get_error(h, stream, flags);
}

int stixels_get_error(stixels_t h, void* stream, uint32_t* flags)
{
    if (!h || !flags) return STIXELS_E_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    uint32_t v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_status(e);
    *flags = v;
    return STIXELS_OK;
}

// The address at which the device reads / writes host memory p, or null if it
// cannot: page-locked host memory is mapped into the device's address space
// under unified addressing (cudaPointerGetAttributes then reports it as host
// memory with a device pointer); pageable memory is not.
static void* device_view(const void* p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();                       // an unknown pointer is not an error here
        return nullptr;
    }
    return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

int stixels_compute_host(stixels_t h, const float* h_disparity, int H, int W, stixel_t* h_stixels,
                         int32_t* h_counts, float* h_cost)
{
    int rc = check_frame(h, H, W);
    if (rc) return rc;
    const FrameGeom g = geom(h, H, W);
    if (g.H == 0 || g.ncols == 0) return STIXELS_OK;
    if (!h_disparity || !h_stixels || !h_counts) return STIXELS_E_INVALID_ARG;
    const size_t in_bytes = sizeof(float) * (size_t)H * W;
    const int cap = h->hm.p.max_stixels_per_col;
    const size_t st_bytes = align_up(sizeof(stixel_t) * (size_t)g.ncols * cap, 256);
    const size_t cnt_bytes = align_up(sizeof(int32_t) * (size_t)g.ncols, 256);
    const size_t cost_bytes = align_up(sizeof(float) * (size_t)g.ncols, 256);
    const size_t out_bytes = st_bytes + cnt_bytes + cost_bytes;
    // Page-locked buffers are used in place over the host link (the reduction
    // reads the frame from host memory once; the DP writes its results there),
    // others through device staging buffers and copies.
    const float* d_in = static_cast<const float*>(device_view(h_disparity));
    stixel_t* d_st = static_cast<stixel_t*>(device_view(h_stixels));
    int32_t* d_cnt = static_cast<int32_t*>(device_view(h_counts));
    float* d_cost = h_cost ? static_cast<float*>(device_view(h_cost)) : nullptr;
    const bool out_mapped = d_st && d_cnt && (!h_cost || d_cost);
    cudaError_t e = cudaSuccess;
    if (!d_in && h->in_bytes < in_bytes) {
        cudaFree(h->d_in);
        h->d_in = nullptr;
        h->in_bytes = 0;
        e = cudaMalloc(&h->d_in, in_bytes);
        if (e != cudaSuccess) return cuda_status(e);
        h->in_bytes = in_bytes;
    }
    if (!out_mapped && h->out_bytes < out_bytes) {
        cudaFree(h->d_out);
        h->d_out = nullptr;
        h->out_bytes = 0;
        e = cudaMalloc(&h->d_out, out_bytes);
        if (e != cudaSuccess) return cuda_status(e);
        h->out_bytes = out_bytes;
    }
    stixels_output_t out;
    if (out_mapped) {
        out.stixels = d_st;
        out.counts = d_cnt;
        out.column_cost = d_cost;
    } else {
        out.stixels = (stixel_t*)h->d_out;
        out.counts = (int32_t*)((char*)h->d_out + st_bytes);
        out.column_cost = (float*)((char*)h->d_out + st_bytes + cnt_bytes);
    }
    out.column_cost_fixed = nullptr;
    out.ncols = g.ncols;
    out.capacity = cap;
    if (!d_in) {
        e = cudaMemcpyAsync(h->d_in, h_disparity, in_bytes, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_status(e);
        d_in = h->d_in;
    }
    // this frame's status flags go straight to the pinned word (cleared here,
    // read after the wait); the handle's own error word is left alone
    volatile uint32_t* flags_word = h->h_err;
    uint32_t* d_flags = static_cast<uint32_t*>(device_view(h->h_err));
    *flags_word = 0;
    rc = compute_frame(h, d_in, H, W, h->stream, &out, d_flags ? d_flags : h->d_err);
    if (rc) {
        // a stage may have been launched before the failing one: let it finish
        // with the caller's buffers before they are handed back
        cudaStreamSynchronize(h->stream);
        return rc;
    }
    if (!out_mapped) {
        e = cudaMemcpyAsync(h_counts, out.counts, sizeof(int32_t) * g.ncols, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_stixels, out.stixels, sizeof(stixel_t) * (size_t)g.ncols * cap,
                                cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && h_cost)
            e = cudaMemcpyAsync(h_cost, out.column_cost, sizeof(float) * g.ncols, cudaMemcpyDeviceToHost, h->stream);
    }
    // (were the word not device-addressable, the flags went to the handle's
    // error word: read and clear it on the same stream, one wait in all)
    if (!d_flags && e == cudaSuccess)
        e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream);
    if (!d_flags && e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const uint32_t flags = *flags_word;
    if (flags & (STIXELS_ERR_INFEASIBLE | STIXELS_ERR_TIMEOUT)) return STIXELS_E_DEVICE_FAULT;
    if (flags & STIXELS_ERR_CAPACITY) return STIXELS_E_CAPACITY;
    return STIXELS_OK;
}

int stixels_model_tables(const stixels_params_t* params, int H, int32_t* k_obj, int32_t* g_obj, int32_t* g_sky,
                         double* fg, int32_t* k_ground, int32_t* thr, int32_t* scalars)
{
    if (!params || H < 0 || H > STIXELS_MAX_HEIGHT) return STIXELS_E_INVALID_ARG;
    HostModel m;
    int rc = build_model(params, &m);
    if (rc) return rc;
    if (m.var_sigma) return STIXELS_E_INVALID_ARG;     // per-disparity / per-row residual tables are not exported
    if (k_obj) memcpy(k_obj, m.k_obj.data(), sizeof(int32_t) * m.k_obj.size());
    if (g_obj) memcpy(g_obj, m.g_obj.data(), sizeof(int32_t) * m.g_obj.size());
    if (g_sky) memcpy(g_sky, m.g_sky.data(), sizeof(int32_t) * m.g_sky.size());
    if (H > 0 && (fg || k_ground || thr)) {
        std::vector<char> block;
        int gw = 0;
        if (!build_rows(m, H, &block, &gw)) return STIXELS_E_INVALID_ARG;
        const double* b = reinterpret_cast<const double*>(block.data());
        if (fg) memcpy(fg, b, sizeof(double) * H);
        if (k_ground) memcpy(k_ground, rows_kg(b, H), sizeof(int32_t) * H);
        if (thr) memcpy(thr, rows_thr(b, H), sizeof(int32_t) * H);
    }
    if (scalars) {
        int32_t* s = scalars;
        s[0] = m.c_out;
        s[1] = m.k_sky;
        for (int c = 0; c < 3; ++c) s[2 + c] = m.first[c];
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < 3; ++q) s[5 + 3 * c + q] = m.trans[c][q];
        s[14] = m.pen_grav;
        s[15] = m.pen_div;
        s[16] = m.pen_ord;
        s[17] = m.ord_off;
    }
    return STIXELS_OK;
}

const char* stixels_last_cuda_error(void) { return stx::t_last_cuda_error_string(); }

const char* stixels_status_string(int status)
{
    switch (status) {
        case STIXELS_OK: return "ok";
        case STIXELS_E_INVALID_ARG: return "invalid argument";
        case STIXELS_E_OOM: return "out of memory";
        case STIXELS_E_CUDA: return "CUDA error";
        case STIXELS_E_CAPACITY: return "stixel capacity exceeded";
        case STIXELS_E_NOT_READY: return "not ready";
        case STIXELS_E_TIMEOUT: return "timeout";
        case STIXELS_E_REJECTED: return "rejected by admission control";
        case STIXELS_E_DEVICE_FAULT: return "device-side error";
        default: return "unknown status";
    }
}

}  // extern "C"
