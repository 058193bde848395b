// noalloc.cu -- stixels_compute_noalloc: the per-frame pipeline without any
// device allocation, for callers that cannot allocate when they process a
// frame (real-time loops, another framework's memory pool, strict budgets,
// code that must not let cudaMalloc / cudaFree synchronise the device).  The
// frame's intermediate buffers live in one fixed array of this file instead of
// the handle's workspace.  The paper has no counterpart of this entry point.
#include "internal.h"

namespace {

// The fixed scratch: part of the library's device image, so every device that
// loads it keeps STIXELS_NOALLOC_SCRATCH_BYTES until the process exits.  Every
// call shares it (calls that overlap on the GPU race).
static __device__ __align__(256) unsigned char g_noalloc_scratch[STIXELS_NOALLOC_SCRATCH_BYTES];

// The array's address on the current device.  In host code g_noalloc_scratch
// is only a host-side stand-in for the symbol, so the device address is
// looked up (which allocates nothing) at every call: a cached address would
// go stale if the device were reset, or the module loaded again in another
// context, and the kernels would then write to memory that is not the array.
int scratch_address(unsigned char** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return stx::status_from_cuda(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
    *out = static_cast<unsigned char*>(p);
    return STIXELS_OK;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int stixels_compute_noalloc(stixels_t h, const float* d_disparity, int H, int W, void* stream,
                                       const stixels_output_t* out)
{
    using namespace stx;
    if (!h || !out || H < 0 || W < 0 || H > STIXELS_MAX_HEIGHT || W > (1 << 24)) return STIXELS_E_INVALID_ARG;
    if (H == 0) return STIXELS_OK;
    HandleView v;
    int rc = handle_view(h, H, &v);            // no row tables for H yet -> INVALID_ARG (would allocate)
    if (rc != STIXELS_OK) return rc;
    if (v.ground_estimate || v.global_map) return STIXELS_E_INVALID_ARG;   // their work does not fit the fixed array
    FrameGeom g;
    g.H = H;
    g.W = W;
    g.s = v.stixel_width;
    g.ncols = W / g.s;
    g.P = lut_pitch(H);
    if (out->ncols != g.ncols || out->capacity != v.capacity) return STIXELS_E_INVALID_ARG;
    if (g.ncols == 0) return STIXELS_OK;
    if (!d_disparity || !out->stixels || !out->counts) return STIXELS_E_INVALID_ARG;

    // intermediate layout inside the scratch array (256-byte aligned parts)
    const int F = v.model.dmax + 1;
    const size_t q_off = 0;
    const size_t pd_off = q_off + round256(sizeof(int16_t) * (size_t)g.ncols * H);
    const size_t lut = round256(sizeof(int32_t) * (size_t)g.ncols * g.P);
    const size_t pg_off = pd_off + lut, ps_off = pg_off + lut, po_off = ps_off + lut;
    const size_t total = po_off + round256(sizeof(int32_t) * (size_t)g.ncols * F * g.P);
    if (total > STIXELS_NOALLOC_SCRATCH_BYTES) return STIXELS_E_INVALID_ARG;   // frame too large for the array

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != v.device) return STIXELS_E_INVALID_ARG;
    unsigned char* base = nullptr;
    rc = scratch_address(&base);
    if (rc != STIXELS_OK) return rc;
    int16_t* q = reinterpret_cast<int16_t*>(base + q_off);
    int32_t* pd = reinterpret_cast<int32_t*>(base + pd_off);
    int32_t* pg = reinterpret_cast<int32_t*>(base + pg_off);
    int32_t* ps = reinterpret_cast<int32_t*>(base + ps_off);
    int32_t* po = reinterpret_cast<int32_t*>(base + po_off);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every byte read below is written earlier in this call: no clearing needed
    cudaError_t e = launch_reduce(d_disparity, g, v.model.dmax, v.reduce_mode, q, st);
    if (e == cudaSuccess) e = launch_luts(q, g, v.model, v.rows, pd, pg, ps, po, st, 1);
    if (e == cudaSuccess) e = launch_dp(pd, pg, ps, po, g, v.model, v.rows, v.rp, v.pixel_floor, *out, v.err, st);
    return status_from_cuda(e);
}
