/*
 * stixels.h -- C ABI of a GB300 (sm_103a) implementation of multi-stixel
 * estimation, the method of "GPU-accelerated real-time stixel computation"
 * (Hernandez-Juarez et al., arXiv 1610.04124).
 *
 * The library takes an FP32 disparity map (e.g. from semi-global matching),
 * reduces every stixel-width column to one pixel per row (Sec. 5.1), builds the
 * per-column cost look-up tables (Sec. 3.4, Sec. 5.2), and solves, per column,
 * the MAP segmentation into ground, object and sky stixels with the dynamic
 * program of Eq. 5-6 (Sec. 3.3, Sec. 5.3), followed by backtracking (Sec. 5.4).
 *
 * Conventions used throughout:
 *   - Image rows: 0 = top row.  Columns are independent (Sec. 3).
 *   - A disparity map is H x W FP32, row-major, contiguous (pitch W).
 *     ncols = floor(W / stixel_width); the last W mod stixel_width pixels of
 *     every row are ignored.
 *   - Disparities are clamped to [0, dmax] (NaN -> 0) and put on a 1/16-pixel
 *     grid ("Q4 code" = round-half-even(16 d)) before any other step.
 *   - The DP decides in exact fixed point: every per-pixel cost term and
 *     every prior is rounded to a multiple of 2^-12 cost units, sums are exact
 *     int32 arithmetic (internal unit 2^-14).  Decisions are therefore
 *     deterministic and independent of thread scheduling, and ties are broken
 *     exactly.  The ground line and the gravity / diving / ordering thresholds
 *     are not rounded.  The reported column cost is the chosen segmentation's
 *     cost in real arithmetic (see stixels_output_t).
 *   - "Device pointer" = memory the CUDA device can address (cudaMalloc,
 *     torch CUDA tensors, managed memory).  Streams are cudaStream_t passed as
 *     void*; NULL = the legacy default stream.
 *
 * Errors: every function returns an int status (enum stixels_status).  No
 * function throws, aborts, or traps on the device.  Kernels that detect a
 * per-column condition (output capacity exceeded, no feasible segmentation)
 * record it in a per-handle device error word that stixels_get_error() reads.
 *
 * Threading: a stixels_t handle is not re-entrant -- do not call compute-type
 * functions on one handle from several host threads at once.  Different
 * handles are independent.  The server functions (stixels_submit/poll) are
 * thread-safe.
 */
#ifndef STIXELS_H
#define STIXELS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STIXELS_ABI_VERSION 2
#define STIXELS_MAX_STIXEL_WIDTH 16
#define STIXELS_MAX_DMAX 255
#define STIXELS_MAX_HEIGHT 2048

/* Status codes. */
enum stixels_status {
    STIXELS_OK = 0,
    STIXELS_E_INVALID_ARG = 1,   /* a parameter or size is out of range (see each function) */
    STIXELS_E_OOM = 2,           /* device or pinned host allocation failed, or over budget */
    STIXELS_E_CUDA = 3,          /* a CUDA runtime call failed (launch, copy, sync) */
    STIXELS_E_CAPACITY = 4,      /* a column had more stixels than the output capacity */
    STIXELS_E_NOT_READY = 5,     /* the ticket's result is not finished yet */
    STIXELS_E_TIMEOUT = 6,       /* a wait ran out of time */
    STIXELS_E_REJECTED = 7,      /* admission refused (no slot / memory budget) */
    STIXELS_E_DEVICE_FAULT = 8   /* a kernel reported an internal error (e.g. infeasible column) */
};

/* Stixel classes (Sec. 3.1); this order is also the tie-break order. */
enum stixels_class { STIXELS_OBJECT = 0, STIXELS_GROUND = 1, STIXELS_SKY = 2 };

/* Bits of the device error word. */
#define STIXELS_ERR_CAPACITY 1u    /* some column's stixel count exceeded the capacity */
#define STIXELS_ERR_INFEASIBLE 2u  /* some column has no finite-cost segmentation */
#define STIXELS_ERR_TIMEOUT 4u     /* an internal wait of a kernel gave up (bounded spin); column left empty */

/*
 * Model parameters (Sec. 3; Eq. 3 for the sensor model; the five prior
 * constraints of Sec. 3: BIC, gravity, ordering, staggering, diving).  The
 * paper takes the prior values from Pfeiffer's thesis, which it does not
 * reproduce; stixels_params_default() returns this library's own defaults.
 * All priors are -ln P costs >= 0; INFINITY marks a forbidden configuration.
 */
typedef struct stixels_params {
    float focal_px;            /* focal length in px (only for reported depth; not used by the DP) */
    float baseline_m;          /* stereo baseline in m */
    float camera_height_m;     /* camera height above the ground plane in m (> 0) */
    float pitch_rad;           /* camera pitch in rad */
    int32_t horizon_row;       /* image row (0 = top) of the horizon */
    int32_t stixel_width;      /* s in [1, STIXELS_MAX_STIXEL_WIDTH] */
    int32_t dmax;              /* largest disparity, [1, STIXELS_MAX_DMAX]; d_range = dmax */
    float p_out;               /* outlier rate of the sensor model, (0, 1) */
    float sigma_ground;        /* disparity noise (px) of each class model, > 0 */
    float sigma_object;
    float sigma_sky;
    float prior_first[3];      /* cost of the class of the bottom stixel: object, ground, sky */
    float prior_trans[3][3];   /* [class above][class below] transition cost */
    float cost_new_stixel;     /* BIC: cost added once per stixel */
    float cost_gravity;        /* object directly above ground, nearer than the ground at its base */
    float eps_gravity;         /*   tolerance (px) */
    float cost_diving;         /* object directly above ground, farther than the ground at its base */
    float eps_diving;          /*   tolerance (px) */
    float cost_order;          /* object directly above an object, nearer than it */
    float eps_order;           /*   tolerance (px) */
    int32_t reduce_mode;       /* 0 = median of the s pixels (default), 1 = mean (paper Sec. 5.1) */
    int32_t max_stixels_per_col; /* output capacity per column, >= 1 */
    int32_t pixel_grid;        /* 0 = reduced disparities on the 1/16-px grid (default); 1 = whole
                                  pixels, the paper's LUT_cost variant (Sec. 3.4): each reduced value
                                  is rounded to the nearest integer (halves up) and the object pixel
                                  costs are read from a (dmax+1) x (dmax+1) table built at create */
    /* Disparity-dependent noise (Eq. 3's sigma^c(f, v), "a sigmoid function"; the
     * paper defers its form to Pfeiffer's thesis, so this is a parameterised
     * logistic): sigma^c(f) = sigma_c * (1 + sigma_gain / (1 + exp(-(f - sigma_mid) /
     * sigma_width))), with f the model disparity (object: its f; ground: the ground
     * line at the row; sky: 0).  sigma_gain = 0 (default) is the constant-sigma model;
     * otherwise sigma_gain in (-1, 10] and sigma_width > 0 (px), and the library keeps
     * one residual table per object disparity and per ground row. */
    float sigma_gain;
    float sigma_mid;
    float sigma_width;
    int32_t ground_estimate;   /* 0 = ground line from the camera parameters (default); 1 = estimated
                                  for every frame from its v-disparity (stixels_estimate_ground), by
                                  stixels_compute / _compute_host and in batches and the server (not
                                  by stixels_compute_noalloc); needs sigma_gain = 0 and
                                  ncols * H <= 7,000,000 */
    int32_t global_map;        /* 0 = the paper's DP (Eq. 6: one best stixel per row and class, so the
                                  ordering prior is judged against that stixel only); 1 = the global MAP
                                  with the ordering prior exact (object states carry their disparity),
                                  by stixels_compute / _compute_host / _solve and in batches and the
                                  server (not by stixels_compute_noalloc); about 8 H (dmax+3) bytes of
                                  workspace per column; a column's shared-memory state, about
                                  28 H + 388 (dmax+1) + 6 KB bytes, fits every height and dmax the
                                  library takes */
} stixels_params_t;

/* One output stixel: 12 bytes. */
typedef struct stixel {
    int16_t row_top;           /* image row of the stixel's top pixel (0 = top of image) */
    int16_t row_bottom;        /* image row of its bottom pixel (row_top <= row_bottom) */
    uint8_t cls;               /* enum stixels_class */
    uint8_t flags;             /* reserved, 0 */
    int16_t reserved;          /* 0 */
    float disparity;           /* exact mean of the stixel's Q4 disparities, in px */
} stixel_t;

/* Output buffers of one frame.  All pointers are device pointers owned by the
 * caller.  stixels: ncols * capacity records, column c at [c * capacity],
 * listed bottom -> top.  counts[c] = number of stixels of column c (it may
 * exceed capacity; then only the bottom `capacity` are written and the error
 * word gets STIXELS_ERR_CAPACITY).  column_cost (optional, may be NULL): the
 * cost of the column's segmentation in real arithmetic -- Eq. 4 per pixel and
 * the priors without the fixed-point grid (per-pixel terms in FP32, summed
 * exactly in fixed point at 2^-24, rounded to FP32 once; within ~3e-7
 * relative of the exact value), over the whole segmentation even when it
 * exceeds capacity.  column_cost_fixed (optional): the DP's fixed-point
 * minimum that chose the segmentation, exactly, as an integer in units of
 * 2^-14. */
typedef struct stixels_output {
    stixel_t* stixels;
    int32_t* counts;
    float* column_cost;
    int32_t* column_cost_fixed;
    int32_t ncols;
    int32_t capacity;
} stixels_output_t;

typedef struct stixels_s* stixels_t;

/* Fill *p with the library's default parameters (320x120 camera of the test
 * workload; adjust the camera fields for your own).  Returns OK, or
 * INVALID_ARG if p is NULL. */
int stixels_params_default(stixels_params_t* p);

/* Create a handle for one camera / parameter set (Sec. 3.4: the offline LUTs
 * -- sensor-model constants and per-class residual tables -- are built here in
 * FP64 and uploaded once to the current CUDA device, where they stay resident).
 * Fails with INVALID_ARG for out-of-range parameters (ranges above; first and
 * transition priors in [0, 1000] or +INFINITY; BIC and the gravity, diving and
 * ordering costs finite in [0, 1000]; eps_gravity, eps_diving in [0, 100];
 * |eps_order| <= 100; the residual tables must reach the outlier cost within
 * dmax px), OOM, or CUDA.  The handle is bound to
 * the device that was current at creation; call it with that device current. */
int stixels_create(const stixels_params_t* params, stixels_t* out_handle);

/* Release the handle and all its device memory.  Waits for work the handle
 * launched to finish.  NULL is accepted. */
int stixels_destroy(stixels_t h);

/* Output shape for an H x W frame: *ncols = floor(W / s), *capacity =
 * max_stixels_per_col. */
int stixels_output_shape(stixels_t h, int H, int W, int* ncols, int* capacity);

/* Pre-allocate the handle's workspace and per-height tables for frames up to
 * H x W, so that later compute calls allocate nothing (and can be captured in a
 * CUDA graph).  Synchronous.  INVALID_ARG if H > STIXELS_MAX_HEIGHT or the
 * fixed-point budget check fails: H * max(C_out, -min K) + 3 * (largest prior
 * of one stixel incl. penalties) must stay below 16384 cost units (about
 * H <= 2000 with the default model). */
int stixels_reserve(stixels_t h, int H, int W);

/*
 * Full pipeline on one frame (Sec. 5.1 -> 5.2 -> 5.3 -> 5.4), asynchronous on
 * `stream`: column reduction + transpose, prefix LUTs, DP + backtracking.
 * d_disparity: device pointer, H x W FP32 row-major; must stay valid until the
 * stream reaches this work.  out: device buffers sized per stixels_output_shape
 * (out->ncols and out->capacity must equal it).  If the workspace is too small
 * it is grown first (a synchronous allocation).  H == 0 or ncols == 0 is a no-op.
 * Returns OK once the kernels are enqueued; per-column conditions are reported
 * through stixels_get_error().
 */
int stixels_compute(stixels_t h, const float* d_disparity, int H, int W, void* stream,
                    const stixels_output_t* out);

/*
 * Same pipeline from HOST memory to HOST memory, synchronous: runs
 * stixels_compute on the handle's own stream and waits.  h_stixels: ncols *
 * capacity records; h_counts: ncols; h_cost (optional): ncols floats.
 * Page-locked (pinned) host buffers are used in place over the host link: the
 * reduction kernel reads a pinned frame directly, and when h_stixels, h_counts
 * and h_cost (if given) are all pinned the DP writes its results into them.
 * Pageable buffers go through device staging buffers and copies (slower).
 * The buffers must not be freed or written by the caller during the call.
 * Returns the compute status, or CAPACITY / DEVICE_FAULT if this frame set a
 * status flag (the flags of this call only; the handle's error word that
 * stixels_get_error reads is not touched).
 */
int stixels_compute_host(stixels_t h, const float* h_disparity, int H, int W,
                         stixel_t* h_stixels, int32_t* h_counts, float* h_cost);

/* Read and clear the handle's device error word (STIXELS_ERR_* bits) after
 * synchronising `stream`. */
int stixels_get_error(stixels_t h, void* stream, uint32_t* flags);

/* Diagnostic for the kernels' failure path (no counterpart in the paper):
 * launches one CTA on `stream` that waits, with the bounded wait every DP
 * kernel uses between its warps, on a flag that nothing sets.  After `polls`
 * polls (1 .. 2^22; each sleeps at most 32 ns) the wait gives up, the kernel
 * records STIXELS_ERR_TIMEOUT in the handle's error word and returns; the
 * call then synchronises `stream` and returns the word in *flags (cleared, as
 * stixels_get_error does).  The context stays usable.  INVALID_ARG for a bad
 * handle, pointer or count. */
int stixels_selftest_wait(stixels_t h, int polls, void* stream, uint32_t* flags);

/* ---- individual stages (the same kernels stixels_compute launches) ---- */

/* Row pitch (in int32 elements) of the prefix LUTs for height H:
 * the smallest multiple of 4 that is >= H + 1. */
int stixels_lut_pitch(int H);

/* Stage 1 (Sec. 5.1): column reduction + transpose.  d_q: device, ncols x H
 * int16 Q4 codes, column c at d_q[c * H + v], v = H-1-r (v = 0 is the bottom
 * image row); with pixel_grid = 1 every code is a multiple of 16. */
int stixels_reduce(stixels_t h, const float* d_disparity, int H, int W, void* stream, int16_t* d_q);

/* The frame's ground line from its v-disparity (the paper assumes the ground
 * slope and horizon known per image, Sec. 3; this is the step before the path),
 * for a handle created with ground_estimate = 1, from the Q4 codes d_q of
 * stixels_reduce.  On the 1/16-px grid: per image row r a histogram of the codes
 * in [16, 16 dmax], smoothed with weights 17 - |t| over |t| <= 16; candidate lines
 * have the code (k (r - h) + 8) >> 4 at rows r > h (slope k / 256 px per row,
 * k = 1..256, horizon at image row h = 0..H-1); a line's votes are the smoothed
 * counts at its codes on the rows where they lie in [16, 16 dmax]; the most
 * votes win, ties to the smaller k, then the smaller h.  d_line (device, 3
 * int32) receives {k, h, votes}; votes = 0 means no ground was seen, and
 * stixels_compute then keeps the camera's line.  INVALID_ARG if the handle
 * was created without ground_estimate, or if ncols * H > 7,000,000. */
int stixels_estimate_ground(stixels_t h, const int16_t* d_q, int H, int ncols, void* stream, int32_t* d_line);

/* Stage 2 (Sec. 3.4, Sec. 5.2): per-column prefix LUTs from Q4 codes d_q
 * (layout of stixels_reduce).  With P = stixels_lut_pitch(H) and F = dmax + 1:
 *   d_pd[c * P + j]             = sum of q over rows v < j           (Q4 units)
 *   d_pg[c * P + j], d_ps[...]  = sum of ground / sky pixel costs over v < j
 *   d_po[(c * F + f) * P + j]   = sum of object pixel costs at integer
 *                                 disparity f over v < j
 * Costs in units of 2^-14 (every pixel cost is a multiple of 4).  Entries
 * j in (H, P) repeat the total.  With pixel_grid = 1 the codes are expected on
 * the whole-pixel grid (multiples of 16, as stixels_reduce writes them); other
 * codes read the table entry of floor(q / 16), clamped to [0, dmax]. */
int stixels_build_luts(stixels_t h, const int16_t* d_q, int H, int ncols, void* stream,
                       int32_t* d_pd, int32_t* d_pg, int32_t* d_ps, int32_t* d_po);

/* Stage 3 (Sec. 3.3, Sec. 5.3-5.4): DP + backtracking from the LUTs of stage 2
 * (same layout); writes `out` as stixels_compute does. */
int stixels_solve(stixels_t h, const int32_t* d_pd, const int32_t* d_pg, const int32_t* d_ps,
                  const int32_t* d_po, int H, int ncols, void* stream, const stixels_output_t* out);

/* Build, on the host only (no CUDA call), the fixed-point model tables that
 * stixels_create would upload for `params`, plus the row tables for height H,
 * into caller-owned host arrays (for inspection and tests).  Returns
 * INVALID_ARG for parameters stixels_create would reject, for H outside
 * [0, STIXELS_MAX_HEIGHT], and for sigma_gain != 0 (whose per-disparity and
 * per-row residual tables are not exported).  Cost values in 2^-14 units, forbidden /
 * infinite entries = 2^29.  Sizes and meaning:
 *   k_obj[dmax+1]    normalisation constant K (Eq. 4) of the object model at integer f
 *   g_obj, g_sky [16*dmax+1]   residual term (e/16)^2 / (2 sigma^2) of the
 *                    object / sky class at Q4 residual e
 *   fg[H]            ground-model disparity f_g(v) (Sec. 3.1) at bottom-up row v,
 *                    in px, unrounded (the ground residual of a pixel is
 *                    (q/16 - fg)^2 / (2 sigma_ground^2) in FP64 on the host,
 *                    then rounded to the cost grid)
 *   k_ground[H]      K of the ground model at row v
 *   thr[H]           gravity / diving thresholds at row v: the object penalty
 *                    applies iff f > (int16)(thr & 0xffff), resp. iff f < thr >> 16
 *   scalars[STIXELS_N_SCALARS] = { C_out, K_sky, first[object, ground, sky],
 *                    trans[above][below] row-major (9), gravity, diving, ordering
 *                    penalties, floor(eps_order) (the ordering penalty applies
 *                    iff f_above > f_below + floor(eps_order)) }
 * Any pointer may be NULL. */
#define STIXELS_N_SCALARS 18
int stixels_model_tables(const stixels_params_t* params, int H, int32_t* k_obj, int32_t* g_obj, int32_t* g_sky,
                         double* fg, int32_t* k_ground, int32_t* thr, int32_t* scalars);

/* ---- batched mode: many frames, one graph-captured launch sequence ---- */

/*
 * A batch is a fixed set of frames -- each with its own camera handle and its
 * own size -- processed together: one launch per pipeline stage covers every
 * column of every frame (columns are independent, Sec. 3), and the DP runs as
 * one persistent kernel whose CTAs take columns from a shared work list,
 * longest first.  The sequence is captured once as a CUDA graph and replayed by
 * stixels_batch_launch.  The batch owns a device input slot and device output
 * buffers per frame; the caller writes frames into the input slots and reads
 * the outputs after the launch completes.  Not part of the paper (an
 * execution mode of the same computation: each frame's results equal
 * stixels_compute's).
 */
typedef struct stixels_batch_s* stixels_batch_t;
typedef struct stixels_frame_desc {
    stixels_t camera;          /* handle whose parameters the frame uses */
    int32_t H, W;              /* frame size, 1 <= H <= STIXELS_MAX_HEIGHT */
} stixels_frame_desc_t;
typedef struct stixels_batch_config {
    int32_t dp_warps;          /* warps per DP CTA: 8 (two CTAs fit an SM) or 16 (one) */
    int32_t dp_ctas_per_sm;    /* persistent DP grid = SMs x this, 1..4 */
} stixels_batch_config_t;

/* Plan a batch: validates every frame, allocates all device memory at once
 * (inputs, intermediates, outputs, work lists), and captures the graph with a
 * default configuration.  The camera handles must outlive the batch.
 * INVALID_ARG (bad frame / handle on another device), OOM, CUDA. */
int stixels_batch_create(const stixels_frame_desc_t* frames, int nframes, stixels_batch_t* out);
/* Device pointer of frame i's input slot (H x W FP32, row-major). */
int stixels_batch_input(stixels_batch_t b, int i, float** d_frame);
/* Device output buffers of frame i (valid until stixels_batch_destroy). */
int stixels_batch_output(stixels_batch_t b, int i, stixels_output_t* out);
/* Copy a frame (H x W FP32, host or device memory) into frame i's input slot,
 * asynchronously on `stream` (cudaMemcpyDefault). */
int stixels_batch_set_input(stixels_batch_t b, int i, const float* src, void* stream);
/* Copy frame i's results out (host or device destinations; any may be NULL):
 * stixels ncols * capacity records, counts / cost / cost_fixed ncols each. */
int stixels_batch_get_output(stixels_batch_t b, int i, stixel_t* stixels, int32_t* counts, float* cost,
                             int32_t* cost_fixed, void* stream);
/* Replay the captured pipeline for all frames on `stream` (asynchronous). */
int stixels_batch_launch(stixels_batch_t b, void* stream);
/* Change the DP launch shape and re-capture the graph (synchronous). */
int stixels_batch_set_config(stixels_batch_t b, const stixels_batch_config_t* cfg);
int stixels_batch_get_config(stixels_batch_t b, stixels_batch_config_t* cfg);
/* Autotuner: times every supported launch shape on this batch (a few
 * launches each, CUDA events on `stream`) and keeps the fastest.  With a cache
 * file (may be NULL), a previous result for the same device and batch shape
 * (the multiset of frame sizes, stixel widths and dmax) is reused instead, and
 * new results are appended.  *chosen (may be NULL) receives the choice. */
int stixels_batch_tune(stixels_batch_t b, void* stream, const char* cache_path, stixels_batch_config_t* chosen);
int stixels_batch_destroy(stixels_batch_t b);

/* ---- serving: continuous batching of frames from many cameras ---- */

/*
 * A server admits frames from any number of camera handles as they arrive and
 * runs them with continuous batching: a scheduler thread takes every admitted
 * frame whose input has been copied in and runs them together as one
 * iteration -- a lone frame below 800 rows through the kernels of
 * stixels_compute, any other set as one batch (the kernels of the batched
 * mode, tables rebuilt per iteration, the DP's launch shape chosen by the
 * iteration's size) -- on one of three CUDA streams whose previous iteration
 * has finished, so frames admitted while iterations are on the GPU start in
 * the next one and up to three overlap on the device.
 * Device memory comes from one arena of mem_budget_bytes allocated at
 * creation: a frame is admitted only if a slot and arena space for its input,
 * intermediates and outputs are free, else stixels_submit returns
 * STIXELS_E_REJECTED at once.  Results are bit-identical to stixels_compute on
 * the same frame alone.  submit and poll are thread-safe.  A camera handle in
 * use by a server must not be used concurrently outside it.
 */
typedef struct stixels_server_s* stixels_server_t;
typedef struct stixels_server_stats {
    uint64_t submitted, admitted, rejected, completed, iterations;
    uint64_t frames_in_iterations;     /* sum of batch sizes (mean batch = this / iterations) */
    uint64_t bytes_in_use, bytes_budget;
    int32_t slots_in_use, max_slots;
} stixels_server_stats_t;

/* Create a server on the current device: allocates the arena (mem_budget_bytes,
 * >= 1 MiB) and starts the scheduler thread.  max_slots in [1, 4096]. */
int stixels_server_create(size_t mem_budget_bytes, int max_slots, stixels_server_t* out);
/* Admit one frame (H x W FP32 in host or device memory) for `camera`: copies it
 * into the server (the caller may reuse the buffer on return) and queues it.
 * *ticket identifies the request.  STIXELS_E_REJECTED if no slot or not enough
 * arena memory is free right now; INVALID_ARG for a bad frame or handle. */
int stixels_submit(stixels_server_t s, stixels_t camera, const float* disparity, int H, int W, uint64_t* ticket);
/* Wait up to timeout_us (0 = just check) for the ticket's result.  On success
 * copies the result into `out` (host or device buffers, ncols / capacity as
 * stixels_output_shape; column_cost, column_cost_fixed optional), frees the
 * frame's slot and retires the ticket.  STIXELS_E_NOT_READY if timeout_us == 0
 * and the frame is not done, STIXELS_E_TIMEOUT if a positive wait ran out,
 * INVALID_ARG for an unknown ticket, a ticket another poll is already
 * copying out, or mismatched buffers. */
int stixels_poll(stixels_server_t s, uint64_t ticket, const stixels_output_t* out, int timeout_us);
int stixels_server_stats(stixels_server_t s, stixels_server_stats_t* stats);
/* Stop the scheduler, wait for frames on the GPU, release everything.  Tickets
 * not yet polled are dropped. */
int stixels_server_destroy(stixels_server_t s);

/*
 * Scratch-free variant of stixels_compute (this library's addition; the paper
 * has no counterpart).  For callers that cannot allocate device memory when
 * they process a frame -- real-time loops where an allocation could stall or
 * fail, code running inside another framework's memory pool or under a strict
 * memory budget, or code that must not synchronise the device the way
 * cudaMalloc / cudaFree can.  Such callers create the handle and call
 * stixels_reserve(h, H, W) once at start-up; stixels_compute_noalloc then
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *
 * Same computation, arguments and output as stixels_compute (device input,
 * device output buffers, asynchronous on `stream`), but the frame's
 * intermediate buffers (reduced column codes and prefix LUTs, the same bytes
 * stixels_compute keeps in the handle's workspace) live in one fixed device
 * array inside the library, STIXELS_NOALLOC_SCRATCH_BYTES large, which every
 * device that loads the library keeps until the process exits.
 *   - Size limit: frames whose intermediates exceed the array (about
 *     ncols * (dmax + 4) * (H + 4) * 4 bytes) are rejected with
 *     STIXELS_E_INVALID_ARG; 1024 x 440 at stixel width 5, dmax 128 fits.
 *   - The handle must already hold the row tables for height H (from
 *     stixels_reserve or an earlier stixels_compute with that height);
 *     otherwise STIXELS_E_INVALID_ARG (creating them would allocate).
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress; it allocates nothing), so a device reset or a
 *     new context is followed; the first call on a device may load the
 *     module there, so make it before any stream capture.
 *   - Every call uses the same array, which keeps the previous call's
 *     contents; the pipeline overwrites every byte it reads, so nothing needs
 *     clearing, but calls whose work overlaps on the same GPU (issued on
 *     different streams or from different host threads) race on it: order
 *     them on one stream or synchronise between them.  Each device has its own
 *     copy of the array.
 */
#define STIXELS_NOALLOC_SCRATCH_BYTES (48u << 20)
int stixels_compute_noalloc(stixels_t h, const float* d_disparity, int H, int W, void* stream,
                            const stixels_output_t* out);

/* Human-readable name of a status code (static storage). */
const char* stixels_status_string(int status);
/* Text of the CUDA error behind this thread's most recent STIXELS_E_CUDA /
 * STIXELS_E_OOM status (static storage; "no error" if none). */
const char* stixels_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STIXELS_H */
