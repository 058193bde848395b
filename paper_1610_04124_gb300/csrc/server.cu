// server.cu -- serving: admission by slots and a device-memory arena, and a
// scheduler thread doing continuous batching over three CUDA streams.
//
// Life of a frame: stixels_submit reserves arena space (input, intermediates,
// outputs) and a status word (page-locked host memory that the kernels set
// through its device mapping), copies the frame in on the copy stream and
// waits for that copy, then queues the request.  The scheduler takes every
// queued request; a lone frame below 800 rows goes through the per-frame
// kernels, any other set gets the batch tables (the planner of the batched
// mode), uploaded through a pinned staging buffer, and the batched kernels.
// Each iteration runs on a compute stream whose previous iteration has
// finished (when all three are busy, on the one launched first, once it is
// done), recording one completion event per iteration: at most three
// iterations are in flight and they overlap on the device, and no iteration
// waits behind a long one while another stream is free.
// stixels_poll checks the request's iteration event, reads its status word,
// copies the results out on the calling thread's stream (one wait) and
// returns the slot's memory and status word.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace stx;

namespace {

constexpr int kStreams = 3;
constexpr size_t kTableBytes = 8u << 20;      // per stream: device tables and pinned staging
constexpr int kMaxBatchFrames = 512;
// frames of this many rows or more are "tall": alone they keep the batched
// kernels, whose 16-warp DP shape suits them (below, a lone frame takes the
// per-frame kernels)
constexpr int kTallRows = 800;

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// First-fit allocator over [0, size) of the arena, 256-byte granules,
// coalescing neighbours on free.
class Arena {
public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = up256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Iteration {
    cudaEvent_t done = nullptr;
    ~Iteration()
    {
        if (done) cudaEventDestroy(done);
    }
};

enum class State { Queued, Running };

struct Request {
    uint64_t ticket = 0;
    FrameJob job;
    size_t off = 0, bytes = 0;
    uint32_t* d_err = nullptr;          // the frame's status word (device view of h_flags[flag])
    int flag = -1;                      // its index in the server's page-locked status words
    State state = State::Queued;
    bool claimed = false;               // a poll is copying its results out
    int status = STIXELS_OK;            // launch failure of its iteration
    std::shared_ptr<Iteration> iter;
};

}  // namespace

struct stixels_server_s {
    int device = 0;
    int max_slots = 0;
    char* d_arena = nullptr;
    std::unique_ptr<Arena> arena;
    cudaStream_t copy_stream = nullptr;
    cudaStream_t streams[kStreams] = {};
    char* d_tables[kStreams] = {};
    char* h_staging[kStreams] = {};
    // per-slot status words in page-locked host memory, mapped for the device:
    // the kernels set a frame's flags there, submit clears them and poll reads
    // them, with no stream operation for either
    uint32_t* h_flags = nullptr;
    uint32_t* d_flags = nullptr;
    std::vector<int> free_flags;
    std::shared_ptr<Iteration> last[kStreams];
    uint64_t launched[kStreams] = {};   // iteration number of each stream's last iteration

    std::mutex mu;
    std::condition_variable cv_work;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> requests;
    std::deque<std::shared_ptr<Request>> queue;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    stixels_server_stats_t stats{};
};

namespace {

int status_of(cudaError_t e) { return status_from_cuda(e); }

void release_request(stixels_server_t s, const std::shared_ptr<Request>& r)
{
    if (r->flag >= 0) s->free_flags.push_back(r->flag);
    r->flag = -1;
    s->arena->release(r->off, r->bytes);
    s->requests.erase(r->ticket);
    s->stats.slots_in_use = (int32_t)s->requests.size();
    s->stats.bytes_in_use = s->arena->used();
}

void scheduler(stixels_server_t s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) return;
            while (!s->queue.empty() && (int)batch.size() < kMaxBatchFrames) {
                batch.push_back(s->queue.front());
                s->queue.pop_front();
            }
        }
        // a stream whose previous iteration is done (its staging and tables
        // are then free); with none, wait for the oldest, which the device
        // took first
        int k = -1;
        for (int q = 0; q < kStreams && k < 0; ++q)
            if (!s->last[q] || cudaEventQuery(s->last[q]->done) == cudaSuccess) k = q;
        if (k < 0) {
            k = 0;
            for (int q = 1; q < kStreams; ++q)
                if (s->launched[q] < s->launched[k]) k = q;
            cudaEventSynchronize(s->last[k]->done);
        }
        // a lone frame below 800 rows runs the per-frame kernels on its own
        // buffers (no tables; a lone 1024x440 frame 121 -> 105 us, 640x240
        // 60 -> 56 us); otherwise plan the iteration, halving it (returning
        // the rest to the queue) while its tables do not fit the staging
        // buffer
        const bool lone = batch.size() == 1 && batch[0]->job.g.H < kTallRows;
        BatchTables t;
        for (; !lone;) {
            std::vector<FrameJob> jobs;
            jobs.reserve(batch.size());
            for (auto& r : batch) jobs.push_back(r->job);
            plan_tables(jobs, &t);
            if (t.host.size() <= kTableBytes || batch.size() == 1) break;
            std::lock_guard<std::mutex> lock(s->mu);
            const size_t keep = batch.size() / 2;
            for (size_t i = batch.size(); i-- > keep;) s->queue.push_front(batch[i]);
            batch.resize(keep);
        }
        auto it = std::make_shared<Iteration>();
        cudaError_t e = cudaEventCreateWithFlags(&it->done, cudaEventDisableTiming);
        if (lone) {
            if (e == cudaSuccess) e = launch_frame_job(batch[0]->job, s->streams[k]);
        } else {
            if (e == cudaSuccess && t.host.size() > kTableBytes) e = cudaErrorInvalidValue;
            if (e == cudaSuccess) {
                memcpy(s->h_staging[k], t.host.data(), t.host.size());
                e = cudaMemcpyAsync(s->d_tables[k], s->h_staging[k], t.host.size(), cudaMemcpyHostToDevice,
                                    s->streams[k]);
            }
        }
        // the DP's launch shape: an iteration that holds a tall frame (800
        // rows or more) and at most three columns per SM runs faster with 16
        // warps per column, one CTA per SM (a lone 2048x880 frame 693 -> 533
        // us); every other one with 8 warps, two CTAs per SM (a lone 1024x440
        // frame 121 us, against 154 us)
        const bool tall = t.maxH >= kTallRows && t.nitems <= 3 * sm_count();
        if (!lone && e == cudaSuccess && t.nlut > 0)
            e = enqueue_tables(t, s->d_tables[k], tall ? 16 : 8, tall ? 1 : 2, s->streams[k]);
        if (e == cudaSuccess) e = cudaEventRecord(it->done, s->streams[k]);
        const int launch_status = e == cudaSuccess ? STIXELS_OK : status_of(e);
        if (e != cudaSuccess && it->done) cudaEventRecord(it->done, s->streams[k]);   // polls must still return
        {
            std::lock_guard<std::mutex> lock(s->mu);
            for (auto& r : batch) {
                r->state = State::Running;
                r->status = launch_status;
                r->iter = it;
            }
            s->stats.iterations += 1;
            s->stats.frames_in_iterations += batch.size();
        }
        s->last[k] = it;
        s->launched[k] = s->stats.iterations;
    }
}

}  // namespace

extern "C" {

int stixels_server_create(size_t mem_budget_bytes, int max_slots, stixels_server_t* out)
{
    if (!out || mem_budget_bytes < (1u << 20) || max_slots < 1 || max_slots > 4096) return STIXELS_E_INVALID_ARG;
    *out = nullptr;
    stixels_server_s* s = new (std::nothrow) stixels_server_s();
    if (!s) return STIXELS_E_OOM;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return STIXELS_E_CUDA; }
    s->max_slots = max_slots;
    mem_budget_bytes = mem_budget_bytes / 256 * 256;
    cudaError_t e = cudaMalloc(&s->d_arena, mem_budget_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < kStreams && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_tables[k], kTableBytes);
        if (e == cudaSuccess) e = cudaHostAlloc(&s->h_staging[k], kTableBytes, cudaHostAllocDefault);
    }
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_flags, sizeof(uint32_t) * max_slots, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->d_flags, s->h_flags, 0);
    if (e == cudaSuccess) e = prepare_dp_kernels();
    if (e == cudaSuccess) e = prepare_ground_kernels();
    if (e == cudaSuccess) e = prepare_map_kernel();
    if (e != cudaSuccess) {
        stixels_server_destroy(s);
        return status_of(e);
    }
    for (int i = max_slots - 1; i >= 0; --i) s->free_flags.push_back(i);
    s->arena.reset(new Arena(mem_budget_bytes));
    s->stats.bytes_budget = mem_budget_bytes;
    s->stats.max_slots = max_slots;
    s->worker = std::thread(scheduler, s);
    *out = s;
    return STIXELS_OK;
}

int stixels_submit(stixels_server_t s, stixels_t camera, const float* disparity, int H, int W, uint64_t* ticket)
{
    if (!s || !camera || !disparity || !ticket || H < 1 || H > STIXELS_MAX_HEIGHT || W < 1 || W > (1 << 24))
        return STIXELS_E_INVALID_ARG;
    auto r = std::make_shared<Request>();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stats.submitted += 1;
        int rc = handle_prepare(camera, H, &r->job.view);
        if (rc != STIXELS_OK) return rc;
        if (r->job.view.device != s->device) return STIXELS_E_INVALID_ARG;
        FrameGeom& g = r->job.g;
        g.H = H; g.W = W; g.s = r->job.view.stixel_width; g.ncols = W / g.s; g.P = lut_pitch(H);
        if ((r->job.view.ground_estimate && !ground_size_ok(g)) ||
            (r->job.view.global_map && !map_fits(H, r->job.view.model.dmax + 1)))
            return STIXELS_E_INVALID_ARG;
        const size_t C = (size_t)g.ncols, cap = (size_t)r->job.view.capacity;
        const size_t in_b = up256(sizeof(float) * (size_t)H * W);
        const size_t work_b = frame_work_bytes(g, r->job.view);
        const size_t out_b = up256(sizeof(stixel_t) * C * cap) + 3 * up256(sizeof(int32_t) * C) + 256;
        r->bytes = in_b + work_b + out_b;
        if ((int)s->requests.size() >= s->max_slots || !s->arena->alloc(r->bytes, &r->off)) {
            s->stats.rejected += 1;
            return STIXELS_E_REJECTED;
        }
        char* base = s->d_arena + r->off;
        r->job.in = (const float*)base;
        frame_work_carve(&r->job, base + in_b);
        char* o = base + in_b + work_b;
        r->job.out.stixels = (stixel_t*)o;                            o += up256(sizeof(stixel_t) * C * cap);
        r->job.out.counts = (int32_t*)o;                              o += up256(sizeof(int32_t) * C);
        r->job.out.column_cost = (float*)o;                           o += up256(sizeof(int32_t) * C);
        r->job.out.column_cost_fixed = (int32_t*)o;                   o += up256(sizeof(int32_t) * C);
        // admission keeps the live requests below max_slots: a word is free
        r->flag = s->free_flags.back();
        s->free_flags.pop_back();
        reinterpret_cast<volatile uint32_t*>(s->h_flags)[r->flag] = 0u;
        r->d_err = s->d_flags + r->flag;
        r->job.view.err = r->d_err;
        r->job.out.ncols = g.ncols;
        r->job.out.capacity = (int32_t)cap;
        r->ticket = s->next_ticket++;
        s->requests[r->ticket] = r;
        s->stats.admitted += 1;
        s->stats.slots_in_use = (int32_t)s->requests.size();
        s->stats.bytes_in_use = s->arena->used();
    }
    // copy the frame in; the caller may reuse its buffer once this returns
    cudaError_t e = cudaMemcpyAsync((void*)r->job.in, disparity, sizeof(float) * (size_t)H * W, cudaMemcpyDefault,
                                    s->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    std::lock_guard<std::mutex> lock(s->mu);
    if (e != cudaSuccess) {
        release_request(s, r);
        return status_of(e);
    }
    s->queue.push_back(r);
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return STIXELS_OK;
}

int stixels_poll(stixels_server_t s, uint64_t ticket, const stixels_output_t* out, int timeout_us)
{
    if (!s || !out || timeout_us < 0) return STIXELS_E_INVALID_ARG;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->requests.find(ticket);
        if (it == s->requests.end()) return STIXELS_E_INVALID_ARG;
        r = it->second;
        if (out->ncols != r->job.out.ncols || out->capacity != r->job.out.capacity) return STIXELS_E_INVALID_ARG;
        if (r->job.out.ncols > 0 && (!out->stixels || !out->counts)) return STIXELS_E_INVALID_ARG;
    }
    // wait for the frame's iteration: first for the scheduler to pick it up,
    // then for its completion event; the first 2 ms yield the core between
    // checks (a frame takes 0.05 - 1 ms), later ones sleep 20 us
    const auto start = std::chrono::steady_clock::now();
    const auto deadline = start + std::chrono::microseconds(timeout_us);
    for (;;) {
        std::shared_ptr<Iteration> iter;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            iter = r->iter;
        }
        if (iter) {
            if (!iter->done) break;                  // its launch failed; status says why
            cudaError_t q = cudaEventQuery(iter->done);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return status_of(q);
        }
        const auto now = std::chrono::steady_clock::now();
        if (now >= deadline) return timeout_us == 0 ? STIXELS_E_NOT_READY : STIXELS_E_TIMEOUT;
        if (now - start < std::chrono::milliseconds(2))
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    {
        // one poll copies a frame out and frees it; a concurrent poll of the
        // same ticket finds it claimed
        std::lock_guard<std::mutex> lock(s->mu);
        if (r->claimed || !s->requests.count(ticket)) return STIXELS_E_INVALID_ARG;
        r->claimed = true;
    }
    const stixels_output_t& src = r->job.out;
    const size_t C = (size_t)src.ncols;
    // the iteration is done: its kernels' writes to the status word are visible
    const uint32_t flags = reinterpret_cast<volatile uint32_t*>(s->h_flags)[r->flag];
    // the results out on this thread's own stream, one wait
    cudaError_t e = cudaSuccess;
    if (C) {
        const cudaStream_t cs = cudaStreamPerThread;
        e = cudaMemcpyAsync(out->stixels, src.stixels, sizeof(stixel_t) * C * src.capacity, cudaMemcpyDefault, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out->counts, src.counts, sizeof(int32_t) * C, cudaMemcpyDefault, cs);
        if (e == cudaSuccess && out->column_cost)
            e = cudaMemcpyAsync(out->column_cost, src.column_cost, sizeof(float) * C, cudaMemcpyDefault, cs);
        if (e == cudaSuccess && out->column_cost_fixed)
            e = cudaMemcpyAsync(out->column_cost_fixed, src.column_cost_fixed, sizeof(int32_t) * C,
                                cudaMemcpyDefault, cs);
        const cudaError_t w = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = w;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    release_request(s, r);
    s->stats.completed += 1;
    if (r->status != STIXELS_OK) return r->status;
    if (e != cudaSuccess) return status_of(e);
    if (flags & (STIXELS_ERR_INFEASIBLE | STIXELS_ERR_TIMEOUT)) return STIXELS_E_DEVICE_FAULT;
    if (flags & STIXELS_ERR_CAPACITY) return STIXELS_E_CAPACITY;
    return STIXELS_OK;
}

int stixels_server_stats(stixels_server_t s, stixels_server_stats_t* stats)
{
    if (!s || !stats) return STIXELS_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    *stats = s->stats;
    return STIXELS_OK;
}

int stixels_server_destroy(stixels_server_t s)
{
    if (!s) return STIXELS_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (int k = 0; k < kStreams; ++k) {
        if (s->streams[k]) cudaStreamSynchronize(s->streams[k]);
    }
    s->requests.clear();
    s->queue.clear();
    for (int k = 0; k < kStreams; ++k) {
        s->last[k].reset();
        if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
        cudaFree(s->d_tables[k]);
        if (s->h_staging[k]) cudaFreeHost(s->h_staging[k]);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    cudaFree(s->d_arena);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
    return STIXELS_OK;
}

}  // extern "C"
