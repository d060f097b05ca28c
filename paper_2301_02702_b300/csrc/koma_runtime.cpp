// Host runtime of libkoma: the C ABI of include/koma.h.
//
// Responsibilities: argument validation, conversion of the phantom to the
// device layout, sequence preprocessing into step records (regime
// classification, FP64 cumulative gradient moments since the last RF step,
// uniform ADC runs, the matrix-form readout plan), device-memory budget,
// launch configuration, and the kernel launches per simulation (Bloch kernel,
// the tensor-core readout when the sequence has matrix-form groups, the
// fixed-order reduction).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <limits>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "koma.h"
#include "koma_internal.h"
#include "koma_host.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kGammaBar = 42.577478518e6;          // Hz/T
constexpr double kGamma = 2.0 * kPi * kGammaBar;       // rad/s/T
constexpr double kLog2e = 1.44269504088896340736;

}  // namespace

struct koma_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;  // phantoms + sequences + scratch
    int sm_count = 0;
    std::string err;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    int* d_status = nullptr;  // [0] device status flags, [1] batch counter of the grouped kernel
    cudaStream_t own_stream = nullptr;
    // uploads (the phantom's copies and conversion, the synchronous copies
    // and memsets): waited for by the host before anything that uses them is
    // launched; high priority, so an upload's small kernels get SMs while
    // another simulation's kernels run
    cudaStream_t up_stream = nullptr;
    cudaEvent_t ev_job = nullptr;  // end of the last batch job's work on own_stream
    cudaMemPool_t pool = nullptr;  // device memory of phantoms, sequences and scratch
    cudaStream_t alloc_stream = nullptr;  // orders the pool's allocations and frees only
    koma_launch_info last{};
    int64_t live_objects = 0;
    // optional kernel timing: events before the Bloch kernel, after it, after
    // the tensor-core readout (right after the Bloch kernel when there is
    // none) and after the reduction
    bool timing = false;
    bool timing_recorded = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool mma_enabled = true;  // koma_set_mma
    bool rf_maps_enabled = true;  // koma_set_rf_maps
    cudaEvent_t ev_maps = nullptr;  // after the map pre-pass (timing)
    bool maps_timed = false;        // the last timed call ran the pre-pass
    // autotuner results by problem shape (see tune_key): launches of a shape
    // tuned once reuse the choice for other phantoms and sequences of that shape
    struct TuneChoice {
        int s, block, tile;  // spins per thread, threads per CTA, records per tile
    };
    std::map<uint64_t, TuneChoice> tune_cache;  // shape key -> choice
    koma::ConvertStatus* d_conv = nullptr;  // checks and extents of the last phantom upload
    koma::ConvertStatus* h_conv = nullptr;  // pinned host copy of *d_conv
    // pinned staging of sequence uploads (grows, kept): the record block is
    // assembled here and copied by DMA
    char* h_stage = nullptr;
    size_t h_stage_bytes = 0;
    // second context of koma_simulate_host_batch (same device and budget)
    koma_ctx* twin = nullptr;
};

struct koma_phantom {
    koma_ctx* ctx = nullptr;
    int64_t n = 0, n_pad = 0, n_groups = 1;
    float* p32 = nullptr;
    double* p64 = nullptr;
    std::vector<int64_t> group_offsets;  // host copy ([n_groups + 1]) when grouped
    size_t bytes = 0;
    // cached CTA tables of the last grouped launch configuration
    int64_t cfg_spc = -1;
    int64_t* d_cta_begin = nullptr;
    int32_t* d_group_cta = nullptr;
    int grid = 0;
    size_t table_bytes = 0;
    // max |x|, |y|, |z| (m) and |df| (Hz) over the spins
    double max_abs[4] = {0, 0, 0, 0};
    double max_pd = 0;
    // work items of the grouped kernel, built for items_s spins per thread:
    // d_items [n_items + 1] first spin of each item, then (same allocation)
    // d_order [n_items] longest first, d_group_item [n_groups + 1]
    // (items_s = 8: the K3z table instead: d_items [n_units + 1] first spin
    // of each unit of up to 8 spins, d_order [n_units] the unit's item (a
    // warp's segment of a group), d_group_item [n_groups + 1])
    int items_s = 0;
    int64_t n_items = 0, n_units = 0;
    int64_t* d_items = nullptr;
    int32_t* d_order = nullptr;
    int32_t* d_group_item = nullptr;
    size_t items_bytes = 0;
    // motion: per-spin constant velocity (koma_phantom_set_motion)
    float* pv32 = nullptr;   // [PV32_N][n_pad] hi/lo
    double* pv64 = nullptr;  // [3][n_pad]
    double max_v[3] = {0, 0, 0};
    bool moving() const { return pv32 != nullptr; }
    // configuration chosen by koma_tune for one sequence
    const koma_sequence* tuned_seq = nullptr;
    int64_t tuned_n_rec = -1;
    int tuned_s = 0, tuned_block = 0, tuned_tile = 0;
    // every group has a single T1 and a single T2 (a dictionary's entries):
    // the grouped kernel evaluates relaxation once per thread
    bool uni_relax = false;
    // p32 / p64 belong to the caller (koma::phantom_from_device): not freed here
    bool borrowed = false;
};

struct koma_sequence {
    koma_ctx* ctx = nullptr;
    koma_sequence_info info{};
    koma::Rec32* r32 = nullptr;  // one allocation: r32, then r64, then rm
    koma::Rec64* r64 = nullptr;  // null when built without the FP64 stream
    koma::RecM* rm = nullptr;    // null when built without the motion stream
    size_t bytes = 0;
    // matrix-form readout tables, in the same device block after the
    // records: groups, runs (n_mma_runs = rows of the E buffer) and the
    // per-sample source map of the reduction
    koma::MmaGroup* d_mma_groups = nullptr;
    koma::MmaRun* d_mma_runs = nullptr;
    uint8_t* d_from_mma = nullptr;
    int32_t n_mma_groups = 0;
    int64_t n_mma_runs = 0;
    int64_t n_mma_snaps = 0;  // rows of the snapshot buffer
    // repeated RF pulses (same device block): one entry per map slot, and the
    // compacted record stream (each mapped run one REC_MAP record)
    koma::RfMapPulse* d_rf_pulses = nullptr;
    int32_t n_rf_maps = 0;
    koma::Rec32* r32c = nullptr;
    int64_t n_rec_c = 0;
    // every RF step has Gz = 0 and every ADC record one sample: with a
    // phantom of isochromats along z only, the dictionary kernel K3z applies
    // and walks its own copy of the stream (r32z, same device block), whose
    // RF records carry the pulse's rotation and whose PREC/ADC records carry
    // -2 pi Kz as one FP32 value; z_kmax = max |Kz| (turns/m) over them
    bool z_dict = false;
    koma::Rec32* r32z = nullptr;
    double z_kmax = 0.0;
};

namespace {

// NVTX range for the scope (a no-op unless a profiler is attached): marks
// uploads, simulations and their host phases on a profiler's timeline.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

koma_status fail(koma_ctx* ctx, koma_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

koma_status cuda_fail(koma_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? KOMA_E_NOMEM : KOMA_E_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

// Makes ctx->device current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Device memory of phantoms, sequences and scratch comes from the context's
// memory pool (allocations stay mapped, so an upload-simulate-free cycle
// does not pay cudaMalloc/cudaFree). Allocations and frees are ordered on a
// stream of their own that carries no other work, and each completes before
// the call returns, so a block can be used from any stream at once. A free
// first waits for the whole device, as cudaFree does (the memory may still
// be read by a kernel on any stream).
koma_status dev_alloc(koma_ctx* ctx, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return KOMA_OK;
    if (ctx->budget && ctx->used + bytes > ctx->budget)
        return fail(ctx, KOMA_E_NOMEM, "%s: %zu bytes would exceed the memory budget (%zu of %zu used)", what,
                    bytes, ctx->used, ctx->budget);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->alloc_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->alloc_stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_fail(ctx, e, what);
    }
    ctx->used += bytes;
    return KOMA_OK;
}

void dev_free(koma_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFreeAsync(p, ctx->alloc_stream);
    cudaStreamSynchronize(ctx->alloc_stream);
    ctx->used -= std::min(ctx->used, bytes);
}

// Host -> device copy that has landed when the call returns. A plain
// cudaMemcpy from pageable memory may return once the data is staged, before
// the DMA into device memory completes, and it runs on the legacy default
// stream, which the library's non-blocking streams do not wait for: a kernel
// launched next on such a stream could read the block before it arrived.
// The copy is therefore ordered on the context's own stream and waited for.
cudaError_t h2d_sync(koma_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->up_stream);
    return e == cudaSuccess ? cudaStreamSynchronize(ctx->up_stream) : e;
}

// Device memset complete on return (same reason as h2d_sync).
cudaError_t memset_sync(koma_ctx* ctx, void* dst, int value, size_t bytes) {
    cudaError_t e = cudaMemsetAsync(dst, value, bytes, ctx->up_stream);
    return e == cudaSuccess ? cudaStreamSynchronize(ctx->up_stream) : e;
}

// Free ordered after the work already enqueued on `st` (the caller knows
// that no other stream uses the block); nothing waits.
void dev_free_on(koma_ctx* ctx, void* p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    cudaFreeAsync(p, st);
    ctx->used -= std::min(ctx->used, bytes);
}

inline void split(double v, float* hi, float* lo) {
    const float h = static_cast<float>(v);
    *hi = h;
    *lo = static_cast<float>(v - static_cast<double>(h));
}

bool finite_or_posinf(double v) { return std::isfinite(v) || (std::isinf(v) && v > 0); }

// Persistent host worker threads for parallel_for: spawning threads costs
// tens of microseconds each, a noticeable share of an upload. One job runs
// at a time; a caller that finds the pool busy runs its job serially.
class HostPool {
  public:
    static HostPool& get() {
        static HostPool pool;
        return pool;
    }
    int workers() const { return static_cast<int>(threads_.size()); }
    // Runs task(t) for t in [0, k) on the workers and the caller; returns
    // false (nothing run) if another job holds the pool.
    bool try_run(int k, const std::function<void(int)>& task) {
        std::unique_lock<std::mutex> job(job_mu_, std::try_to_lock);
        if (!job.owns_lock()) return false;
        {
            std::lock_guard<std::mutex> lock(mu_);
            task_ = &task;
            n_tasks_ = k;
            next_ = 1;  // task 0 runs on the caller
            done_ = 0;
            ++epoch_;
        }
        cv_.notify_all();
        task(0);
        work_loop_caller();
        std::unique_lock<std::mutex> lock(mu_);
        done_cv_.wait(lock, [&] { return done_ == n_tasks_ - 1; });
        task_ = nullptr;
        return true;
    }

  private:
    HostPool() {
        const unsigned hw = std::max(1u, std::min(std::thread::hardware_concurrency(), 16u));
        for (unsigned i = 1; i < hw; ++i) threads_.emplace_back([this] { worker(); });
    }
    ~HostPool() {
        {
            std::lock_guard<std::mutex> lock(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : threads_) t.join();
    }
    // claim and run tasks of the current job; returns when none are left
    void drain(std::unique_lock<std::mutex>& lock) {
        while (task_ && next_ < n_tasks_) {
            const int t = next_++;
            const std::function<void(int)>* fn = task_;
            lock.unlock();
            (*fn)(t);
            lock.lock();
            if (++done_ == n_tasks_ - 1) done_cv_.notify_all();
        }
    }
    void work_loop_caller() {
        std::unique_lock<std::mutex> lock(mu_);
        drain(lock);
    }
    void worker() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lock(mu_);
        for (;;) {
            cv_.wait(lock, [&] { return stop_ || epoch_ != seen; });
            if (stop_) return;
            seen = epoch_;
            drain(lock);
        }
    }
    std::vector<std::thread> threads_;
    std::mutex job_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int)>* task_ = nullptr;
    int n_tasks_ = 0, next_ = 0, done_ = 0;
    uint64_t epoch_ = 0;
    bool stop_ = false;
};

// Whether this thread's host work may use the worker pool (threads that
// already run side by side, like the server's, keep theirs serial).
thread_local bool t_host_parallel = true;

// (defined with the record builder below)
int n_workers_for(int k);
void run_tasks(int k, const std::function<void(int)>& run);

// fn(lo, hi) over [0, n) split across host threads for large n.
template <class Fn>
void parallel_for(int64_t n, Fn&& fn) {
    const int64_t grain = 1 << 15;
    unsigned hw = std::thread::hardware_concurrency();
    int64_t k = std::min<int64_t>(std::max(1u, std::min(hw, 16u)), (n + grain - 1) / grain);
    if (k <= 1 || !t_host_parallel) {
        fn(int64_t(0), n);
        return;
    }
    const std::function<void(int)> task = [&](int t) { fn(n * t / k, n * (t + 1) / k); };
    if (HostPool::get().try_run(static_cast<int>(k), task)) return;
    // the pool is busy with another caller's job (several threads submitting
    // at once): serial here, so the callers do not oversubscribe the cores
    fn(int64_t(0), n);
}

// Per-spin value checks shared by phantom uploads and server requests.
bool check_spin_values(int64_t n, const double* x, const double* y, const double* z, const double* pd,
                       const double* t1, const double* t2, const double* dw, std::string& msg) {
    char buf[160];
    for (int64_t j = 0; j < n; ++j) {
        if (!std::isfinite(x[j]) || !std::isfinite(y[j]) || !std::isfinite(z[j]) || !std::isfinite(dw[j])) {
            snprintf(buf, sizeof(buf), "phantom: non-finite position/off-resonance at spin %lld", static_cast<long long>(j));
            msg = buf;
            return false;
        }
        if (!std::isfinite(pd[j]) || pd[j] < 0) {
            snprintf(buf, sizeof(buf), "phantom: pd[%lld] = %g", static_cast<long long>(j), pd[j]);
            msg = buf;
            return false;
        }
        if (!finite_or_posinf(t1[j]) || !(t1[j] > 0) || !finite_or_posinf(t2[j]) || !(t2[j] > 0)) {
            snprintf(buf, sizeof(buf), "phantom: T1/T2 of spin %lld must be > 0 (or +inf)", static_cast<long long>(j));
            msg = buf;
            return false;
        }
    }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" double koma_gamma(void) { return kGamma; }

extern "C" const char* koma_version(void) { return "koma-b300 0.1 (sm_103a)"; }

extern "C" koma_status koma_init(int device, size_t mem_budget_bytes, koma_ctx** out) {
    if (!out || device < 0) return KOMA_E_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device >= count) {
        cudaGetLastError();
        return KOMA_E_CUDA;
    }
    koma_ctx* ctx = new (std::nothrow) koma_ctx();
    if (!ctx) return KOMA_E_NOMEM;
    ctx->device = device;
    ctx->budget = mem_budget_bytes;
    int prio_least = 0, prio_greatest = 0;
    DeviceGuard g(device);
    if (!g.ok || cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&ctx->d_status), 2 * sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ctx->up_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        memset_sync(ctx, ctx->d_status, 0, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
        if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
        delete ctx;
        return KOMA_E_CUDA;
    }
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaError_t e = cudaMemPoolCreate(&ctx->pool, &props);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->alloc_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            uint64_t keep = ~0ull;  // keep freed blocks mapped for reuse
            e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (ctx->alloc_stream) cudaStreamDestroy(ctx->alloc_stream);
            if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
            cudaStreamDestroy(ctx->own_stream);
            cudaStreamDestroy(ctx->up_stream);
            cudaFree(ctx->d_status);
            delete ctx;
            return KOMA_E_CUDA;
        }
    }
    *out = ctx;
    return KOMA_OK;
}

extern "C" koma_status koma_destroy(koma_ctx* ctx) {
    if (!ctx) return KOMA_OK;
    if (ctx->live_objects > 0)
        return fail(ctx, KOMA_E_BUSY, "koma_destroy: %lld phantoms/sequences still allocated",
                    static_cast<long long>(ctx->live_objects));
    if (ctx->twin) {
        const koma_status tw = koma_destroy(ctx->twin);
        if (tw != KOMA_OK) return fail(ctx, tw, "koma_destroy: batch context: %s", ctx->twin->err.c_str());
        ctx->twin = nullptr;
    }
    DeviceGuard g(ctx->device);
    for (cudaEvent_t& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->ev_maps) cudaEventDestroy(ctx->ev_maps);
    if (ctx->scratch) dev_free(ctx, ctx->scratch, ctx->scratch_bytes);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->ev_job) cudaEventDestroy(ctx->ev_job);
    if (ctx->alloc_stream) cudaStreamDestroy(ctx->alloc_stream);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->d_conv) cudaFree(ctx->d_conv);
    if (ctx->h_conv) cudaFreeHost(ctx->h_conv);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return KOMA_OK;
}

extern "C" const char* koma_last_error(const koma_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" size_t koma_mem_used(const koma_ctx* ctx) { return ctx ? ctx->used : 0; }

// ---------------------------------------------------------------------------
// phantom
// ---------------------------------------------------------------------------
namespace {

// First half of a phantom upload: argument checks, device blocks, the copies
// of the caller's rows and the conversion kernel, all enqueued on up_stream;
// the conversion's status is copied back into ctx->h_conv (pinned). The
// caller may do other host work before phantom_upload_finish. The FP64 block
// receives the caller's rows [x, y, z, dw, T1, T2, pd] as they are (pinned
// rows are copied by DMA directly; for pageable ones the driver's pipelined
// copy measured faster than packing into pinned memory on the host first);
// the kernel checks every spin, takes the extents, builds the FP32 block,
// turns dw into df and fills the padding.
koma_status phantom_upload_start(koma_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
                                 const double* pd, const double* t1, const double* t2, const double* dw,
                                 const int64_t* group_offsets, int64_t n_groups, koma_phantom** out) {
    if (!out) return fail(ctx, KOMA_E_INVALID, "phantom_upload: out is NULL");
    *out = nullptr;
    if (n < 0) return fail(ctx, KOMA_E_INVALID, "phantom_upload: n = %lld < 0", static_cast<long long>(n));
    if (n > 0 && (!x || !y || !z || !pd || !t1 || !t2 || !dw))
        return fail(ctx, KOMA_E_INVALID, "phantom_upload: NULL array");
    if (group_offsets) {
        if (n_groups < 1) return fail(ctx, KOMA_E_INVALID, "phantom_upload: n_groups < 1");
        if (group_offsets[0] != 0 || group_offsets[n_groups] != n)
            return fail(ctx, KOMA_E_INVALID, "phantom_upload: group_offsets must run from 0 to n");
        for (int64_t g = 0; g < n_groups; ++g)
            if (group_offsets[g + 1] < group_offsets[g])
                return fail(ctx, KOMA_E_INVALID, "phantom_upload: group_offsets decrease at %lld",
                            static_cast<long long>(g));
    } else if (n_groups != 1 && n_groups != 0) {
        return fail(ctx, KOMA_E_INVALID, "phantom_upload: n_groups = %lld without group_offsets",
                    static_cast<long long>(n_groups));
    }
    koma_phantom* ph = new (std::nothrow) koma_phantom();
    if (!ph) return fail(ctx, KOMA_E_NOMEM, "phantom_upload: host allocation");
    ph->ctx = ctx;
    ph->n = n;
    ph->n_pad = std::max<int64_t>(32, (n + 31) / 32 * 32);
    ph->n_groups = group_offsets ? n_groups : 1;
    if (group_offsets) ph->group_offsets.assign(group_offsets, group_offsets + n_groups + 1);
    const int64_t np = ph->n_pad;

    DeviceGuard g(ctx->device);
    const size_t b32 = static_cast<size_t>(koma::P32_N * np) * sizeof(float),
                 b64 = static_cast<size_t>(koma::P64_N * np) * sizeof(double);
    koma_status st = dev_alloc(ctx, reinterpret_cast<void**>(&ph->p32), b32, "phantom_upload");
    if (st == KOMA_OK) st = dev_alloc(ctx, reinterpret_cast<void**>(&ph->p64), b64, "phantom_upload");
    if (st == KOMA_OK && !ctx->d_conv) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ctx->d_conv), sizeof(koma::ConvertStatus));
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&ctx->h_conv), sizeof(koma::ConvertStatus),
                                                cudaHostAllocDefault);
        if (e != cudaSuccess) {
            if (ctx->d_conv) cudaFree(ctx->d_conv);
    if (ctx->h_conv) cudaFreeHost(ctx->h_conv);
            ctx->d_conv = nullptr;
            ctx->h_conv = nullptr;
            st = cuda_fail(ctx, e, "phantom_upload: status word");
        }
    }
    {
        const double* rows[koma::P64_N] = {x, y, z, dw, t1, t2, pd};  // the order of enum P64
        for (int r = 0; r < koma::P64_N && st == KOMA_OK && n > 0; ++r) {
            cudaError_t e = cudaMemcpyAsync(ph->p64 + r * np, rows[r], static_cast<size_t>(n) * sizeof(double),
                                            cudaMemcpyHostToDevice, ctx->up_stream);
            if (e != cudaSuccess) st = cuda_fail(ctx, e, "phantom_upload: copy");
        }
    }
    if (st == KOMA_OK) {
        cudaError_t ce = cudaMemsetAsync(ctx->d_conv, 0, sizeof(koma::ConvertStatus), ctx->up_stream);
        if (ce == cudaSuccess)
            ce = cudaMemsetAsync(&ctx->d_conv->first_bad, 0xff, sizeof(unsigned long long), ctx->up_stream);
        if (ce == cudaSuccess)
            ce = static_cast<cudaError_t>(koma::launch_phantom_convert(ph->p64, ph->p32, n, np, ctx->d_conv,
                                                                       ctx->up_stream));
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(ctx->h_conv, ctx->d_conv, sizeof(koma::ConvertStatus), cudaMemcpyDeviceToHost,
                                 ctx->up_stream);
        if (ce != cudaSuccess) st = cuda_fail(ctx, ce, "phantom_upload: conversion");
    }
    if (st != KOMA_OK) {
        cudaStreamSynchronize(ctx->up_stream);  // no copy may still read or write the blocks
        dev_free(ctx, ph->p32, b32);
        dev_free(ctx, ph->p64, b64);
        delete ph;
        return st;
    }
    // while the rows travel: does every group have a single T1 and T2 (in
    // slices of groups for large phantoms)?
    if (group_offsets) {
        const int k = n >= (int64_t{1} << 20) ? n_workers_for(16) : 1;
        std::vector<uint8_t> uni(static_cast<size_t>(k), 1);
        run_tasks(k, [&](int w) {
            bool u = true;
            for (int64_t gi = n_groups * w / k; gi < n_groups * (w + 1) / k && u; ++gi)
                for (int64_t j = group_offsets[gi] + 1; j < group_offsets[gi + 1] && u; ++j)
                    u = t1[j] == t1[group_offsets[gi]] && t2[j] == t2[group_offsets[gi]];
            uni[w] = u;
        });
        ph->uni_relax = std::find(uni.begin(), uni.end(), 0) == uni.end();
    }
    ph->bytes = b32 + b64;
    ctx->live_objects++;
    *out = ph;
    return KOMA_OK;
}

// Second half: wait for the conversion and check its result. On invalid
// input the phantom is freed, *out reset, and the caller's rows are scanned
// on the host for the message.
koma_status phantom_upload_finish(koma_ctx* ctx, koma_phantom** out, const double* x, const double* y,
                                  const double* z, const double* pd, const double* t1, const double* t2,
                                  const double* dw) {
    koma_phantom* ph = *out;
    DeviceGuard g(ctx->device);
    cudaError_t ce = cudaStreamSynchronize(ctx->up_stream);
    koma_status st = ce == cudaSuccess ? KOMA_OK : cuda_fail(ctx, ce, "phantom_upload: conversion");
    if (st == KOMA_OK && ctx->h_conv->first_bad != ~0ull) {  // report the first offending spin
        std::string msg;
        check_spin_values(ph->n, x, y, z, pd, t1, t2, dw, msg);
        st = fail(ctx, KOMA_E_INVALID, "%s", msg.c_str());
    }
    if (st != KOMA_OK) {
        koma_phantom_free(ph);
        *out = nullptr;
        return st;
    }
    for (int d = 0; d < 4; ++d) {
        double v;
        std::memcpy(&v, &ctx->h_conv->max_bits[d], sizeof(v));
        ph->max_abs[d] = v;
    }
    std::memcpy(&ph->max_pd, &ctx->h_conv->max_bits[4], sizeof(ph->max_pd));
    return KOMA_OK;
}

}  // namespace

extern "C" koma_status koma_phantom_upload(koma_ctx* ctx, int64_t n, const double* x, const double* y,
                                           const double* z, const double* pd, const double* t1,
                                           const double* t2, const double* dw, const int64_t* group_offsets,
                                           int64_t n_groups, koma_phantom** out) {
    NvtxRange nvtx_("koma_phantom_upload");
    if (!ctx) return KOMA_E_INVALID;
    koma_status st = phantom_upload_start(ctx, n, x, y, z, pd, t1, t2, dw, group_offsets, n_groups, out);
    if (st != KOMA_OK) return st;
    return phantom_upload_finish(ctx, out, x, y, z, pd, t1, t2, dw);
}

extern "C" int64_t koma_phantom_n_spins(const koma_phantom* ph) { return ph ? ph->n : -1; }
extern "C" int64_t koma_phantom_n_groups(const koma_phantom* ph) { return ph ? ph->n_groups : -1; }

extern "C" koma_status koma_phantom_free(koma_phantom* ph) {
    if (!ph) return KOMA_OK;
    koma_ctx* ctx = ph->ctx;
    DeviceGuard g(ctx->device);
    if (!ph->borrowed) {
        dev_free(ctx, ph->p32, static_cast<size_t>(koma::P32_N * ph->n_pad) * sizeof(float));
        dev_free(ctx, ph->p64, static_cast<size_t>(koma::P64_N * ph->n_pad) * sizeof(double));
    }
    if (ph->d_cta_begin) dev_free(ctx, ph->d_cta_begin, ph->table_bytes);
    if (ph->d_items) dev_free(ctx, ph->d_items, ph->items_bytes);
    dev_free(ctx, ph->pv32, static_cast<size_t>(koma::PV32_N * ph->n_pad) * sizeof(float));
    dev_free(ctx, ph->pv64, static_cast<size_t>(3 * ph->n_pad) * sizeof(double));
    ctx->live_objects--;
    delete ph;
    return KOMA_OK;
}

extern "C" koma_status koma_phantom_set_motion(koma_phantom* ph, const double* vx, const double* vy,
                                               const double* vz) {
    NvtxRange nvtx_("koma_phantom_set_motion");
    if (!ph) return KOMA_E_INVALID;
    koma_ctx* ctx = ph->ctx;
    const int64_t n = ph->n, np = ph->n_pad;
    const size_t bv32 = static_cast<size_t>(koma::PV32_N * np) * sizeof(float),
                 bv64 = static_cast<size_t>(3 * np) * sizeof(double);
    DeviceGuard g(ctx->device);
    if (!vx && !vy && !vz) {  // back to a static phantom
        dev_free(ctx, ph->pv32, bv32);
        dev_free(ctx, ph->pv64, bv64);
        ph->pv32 = nullptr;
        ph->pv64 = nullptr;
        ph->bytes = static_cast<size_t>(koma::P32_N * np) * sizeof(float) +
                    static_cast<size_t>(koma::P64_N * np) * sizeof(double);
        for (double& m : ph->max_v) m = 0.0;
        return KOMA_OK;
    }
    if (n > 0 && (!vx || !vy || !vz))
        return fail(ctx, KOMA_E_INVALID, "phantom_set_motion: give all three velocity arrays or none");
    for (int64_t j = 0; j < n; ++j)
        if (!std::isfinite(vx[j]) || !std::isfinite(vy[j]) || !std::isfinite(vz[j]))
            return fail(ctx, KOMA_E_INVALID, "phantom_set_motion: non-finite velocity at spin %lld",
                        static_cast<long long>(j));
    std::vector<float> h32(static_cast<size_t>(koma::PV32_N * np), 0.f);
    std::vector<double> h64(static_cast<size_t>(3 * np), 0.0);
    double mv[3] = {0, 0, 0};
    const double* v[3] = {vx, vy, vz};
    for (int d = 0; d < 3; ++d)
        for (int64_t j = 0; j < n; ++j) {
            split(v[d][j], &h32[(2 * d) * np + j], &h32[(2 * d + 1) * np + j]);
            h64[d * np + j] = v[d][j];
            mv[d] = std::max(mv[d], std::fabs(v[d][j]));
        }
    if (!ph->pv32) {
        koma_status st = dev_alloc(ctx, reinterpret_cast<void**>(&ph->pv32), bv32, "phantom_set_motion");
        if (st == KOMA_OK) st = dev_alloc(ctx, reinterpret_cast<void**>(&ph->pv64), bv64, "phantom_set_motion");
        if (st != KOMA_OK) {
            dev_free(ctx, ph->pv32, bv32);
            ph->pv32 = nullptr;
            ph->pv64 = nullptr;
            return st;
        }
        ph->bytes += bv32 + bv64;
    }
    cudaError_t e = h2d_sync(ctx, ph->pv32, h32.data(), bv32);
    if (e == cudaSuccess) e = h2d_sync(ctx, ph->pv64, h64.data(), bv64);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "phantom_set_motion: copy");
    for (int d = 0; d < 3; ++d) ph->max_v[d] = mv[d];
    return KOMA_OK;
}

// ---------------------------------------------------------------------------
// sequence preprocessing
// ---------------------------------------------------------------------------
namespace {

struct RecordBuilder {
    std::vector<koma::Rec32> r32;
    std::vector<koma::Rec64> r64;
    std::vector<koma::RecM> rm;  // motion records (Rec32 fields + first moments)
    bool want64 = true, wantM = true;  // build the FP64 / motion streams too
    int64_t n_adc = 0;
    int64_t n_runs = 0;
    int64_t n_mat = 0;
    // open ADC run (relative to the current t_ref)
    bool run_open = false;
    int64_t run_k0 = 0;
    int run_count = 0;
    double run_k[3] = {0, 0, 0}, run_k1[3] = {0, 0, 0}, run_tau = 0;  // first sample
    double run_dk[3] = {0, 0, 0}, run_dk1[3] = {0, 0, 0}, run_dtau = 0;  // first spacing (count >= 2)
    double last_k[3] = {0, 0, 0}, last_k1[3] = {0, 0, 0}, last_tau = 0;

    // Empty, for a new sequence; the vectors keep their capacity (a builder
    // reused by one thread writes warm memory).
    void reset(bool w64, bool wM) {
        r32.clear();
        r64.clear();
        rm.clear();
        want64 = w64;
        wantM = wM;
        n_adc = n_runs = n_mat = 0;
        run_open = false;
        run_k0 = 0;
        run_count = 0;
        run_tau = run_dtau = last_tau = 0;
        for (int d = 0; d < 3; ++d) run_k[d] = run_k1[d] = run_dk[d] = run_dk1[d] = last_k[d] = last_k1[d] = 0;
    }
    // Motion record carrying `a`'s fields.
    static koma::RecM extend(const koma::Rec32& a) {
        koma::RecM m{};
        m.type = a.type;
        m.count = a.count;
        m.k0 = a.k0;
        for (int i = 0; i < 12; ++i) m.a[i] = a.a[i];
        return m;
    }

    // K1 term bits (4..6) of a motion record whose K1 hi/lo starts at a[off]
    static int k1_bits(const koma::RecM& m, int off) {
        int b = 0;
        for (int d = 0; d < 3; ++d)
            if (m.a[off + 2 * d] != 0.f || m.a[off + 2 * d + 1] != 0.f) b |= 1 << (4 + d);
        return b;
    }

    void close_run() {
        if (!run_open) return;
        koma::Rec32 a{};
        a.type = koma::REC_ADC;
        a.k0 = run_k0;
        for (int d = 0; d < 3; ++d) {
            split(run_k[d], &a.a[2 * d], &a.a[2 * d + 1]);
            a.a[8 + d] = static_cast<float>(run_count > 1 ? run_dk[d] : 0.0);
        }
        split(run_tau, &a.a[6], &a.a[7]);
        a.a[11] = static_cast<float>(run_count > 1 ? run_dtau : 0.0);
        a.count = run_count | (term_bits(a) << koma::kTermShift);
        r32.push_back(a);
        if (want64) {
            koma::Rec64 b{};
            b.type = koma::REC_ADC;
            b.count = run_count;
            b.k0 = run_k0;
            for (int d = 0; d < 3; ++d) {
                b.a[d] = run_k[d];
                b.a[4 + d] = run_count > 1 ? run_dk[d] : 0.0;
                b.a[8 + d] = run_k1[d];
                b.a[11 + d] = run_count > 1 ? run_dk1[d] : 0.0;
            }
            b.a[3] = run_tau;
            b.a[7] = run_count > 1 ? run_dtau : 0.0;
            r64.push_back(b);
        }
        if (wantM) {
            koma::RecM m = extend(a);
            for (int d = 0; d < 3; ++d) {
                split(run_k1[d], &m.a[12 + 2 * d], &m.a[13 + 2 * d]);
                split(run_count > 1 ? run_dk1[d] : 0.0, &m.a[18 + 2 * d], &m.a[19 + 2 * d]);
            }
            m.count = a.count | (k1_bits(m, 12) << koma::kTermShift);
            rm.push_back(m);
        }
        ++n_runs;
        run_open = false;
    }

    static bool close_to(double a, double b, double tol) { return std::fabs(a - b) <= tol; }

    // which phase terms of a PREC/ADC record are nonzero (bit 0..2: K x, y,
    // z; bit 3: tau), from its FP32 hi/lo values
    static int term_bits(const koma::Rec32& a) {
        int m = 0;
        for (int d = 0; d < 4; ++d)
            if (a.a[2 * d] != 0.f || a.a[2 * d + 1] != 0.f) m |= 1 << d;
        return m;
    }

    // Give the first record of every run of consecutive RF records the run's
    // length and maxima (the kernel chooses its rotation path once per run);
    // motion records also get the run's latest midpoint time.
    void mark_rf_runs() {
        size_t i = 0;
        while (i < r32.size()) {
            if (r32[i].type != koma::REC_RF) {
                ++i;
                continue;
            }
            size_t j = i;
            float mb = 0.f, mg[3] = {0.f, 0.f, 0.f}, mdt = 0.f, mt = 0.f;
            while (j < r32.size() && r32[j].type == koma::REC_RF) {
                const koma::Rec32& q = r32[j];
                mb = std::max(mb, std::sqrt(q.a[3] * q.a[3] + q.a[4] * q.a[4]));
                for (int d = 0; d < 3; ++d) mg[d] = std::max(mg[d], std::fabs(q.a[d]));
                mdt = std::max(mdt, q.a[6]);
                if (wantM) mt = std::max(mt, rm[j].a[13]);
                ++j;
            }
            koma::Rec32& h = r32[i];
            h.count = static_cast<int32_t>(std::min<size_t>(j - i, 0x7fffffff));
            h.a[7] = mb * (1.f + 1e-6f);
            for (int d = 0; d < 3; ++d) h.a[8 + d] = mg[d];
            h.a[11] = mdt;
            if (wantM) {
                koma::RecM& hm = rm[i];
                hm.count = h.count;
                for (int k = 7; k < 12; ++k) hm.a[k] = h.a[k];
                hm.a[12] = mt * (1.f + 1e-6f);
            }
            i = j;
        }
    }

    // A sample at (K, K1, tau) relative to t_ref.
    void sample(const double k[3], const double k1[3], double tau) {
        bool joined = false;
        if (run_open && run_count < koma::kMaxAdcRun) {
            const double dk[3] = {k[0] - last_k[0], k[1] - last_k[1], k[2] - last_k[2]};
            const double dk1[3] = {k1[0] - last_k1[0], k1[1] - last_k1[1], k1[2] - last_k1[2]};
            const double dtau = tau - last_tau;
            if (run_count == 1) {
                for (int d = 0; d < 3; ++d) {
                    run_dk[d] = dk[d];
                    run_dk1[d] = dk1[d];
                }
                run_dtau = dtau;
                joined = true;
            } else {
                // uniform spacing: the per-sample rotator reproduces these
                // samples to well below FP32 resolution
                const double ktol = 1e-10 + 1e-12 * (std::fabs(run_dk[0]) + std::fabs(run_dk[1]) +
                                                    std::fabs(run_dk[2]));
                joined = close_to(dk[0], run_dk[0], ktol) && close_to(dk[1], run_dk[1], ktol) &&
                         close_to(dk[2], run_dk[2], ktol) &&
                         close_to(dtau, run_dtau, 1e-15 + 1e-12 * std::fabs(run_dtau));
                // first moments: interval l = run_count - 1 adds dK1_0 + l dtau dK
                const double k1tol = 1e-10 + 1e-12 * (std::fabs(k1[0]) + std::fabs(k1[1]) + std::fabs(k1[2]));
                const double l = static_cast<double>(run_count - 1);
                for (int d = 0; d < 3 && joined; ++d)
                    joined = close_to(dk1[d], run_dk1[d] + l * run_dtau * run_dk[d], k1tol);
            }
        }
        if (joined) {
            ++run_count;
        } else {
            close_run();
            run_open = true;
            run_k0 = n_adc;
            run_count = 1;
            for (int d = 0; d < 3; ++d) {
                run_k[d] = k[d];
                run_k1[d] = k1[d];
            }
            run_tau = tau;
        }
        for (int d = 0; d < 3; ++d) {
            last_k[d] = k[d];
            last_k1[d] = k1[d];
        }
        last_tau = tau;
        ++n_adc;
    }
};

// Moments since t_ref and step counts of a build (FP64).
struct BuildCounts {
    double K[3] = {0, 0, 0}, K1[3] = {0, 0, 0}, tau = 0.0;
    int64_t n_rf = 0, n_precess = 0;
};

// Steps [a, b) into rb, from the state in c at absolute time t0. The sample
// of time point a belongs to the caller (the previous chunk, or the start).
void build_steps(int64_t n_begin, int64_t n_end, double t0, const double* dt, const double* gx, const double* gy,
                 const double* gz, const double* b1_re, const double* b1_im, const uint8_t* adc,
                 RecordBuilder& rb, BuildCounts& c) {
    double t = t0;
    for (int64_t n = n_begin; n < n_end; ++n) {
        const double gm[3] = {0.5 * (gx[n] + gx[n + 1]), 0.5 * (gy[n] + gy[n + 1]), 0.5 * (gz[n] + gz[n + 1])};
        const bool rf = b1_re[n] != 0.0 || b1_im[n] != 0.0;
        const double t_next = t + dt[n];
        if (rf) {
            ++c.n_rf;
            rb.close_run();
            if (c.tau > 0.0) {  // bring the state to the start of this RF step
                koma::Rec32 a{};
                a.type = koma::REC_PREC;
                for (int d = 0; d < 3; ++d) split(c.K[d], &a.a[2 * d], &a.a[2 * d + 1]);
                split(c.tau, &a.a[6], &a.a[7]);
                a.count = RecordBuilder::term_bits(a) << koma::kTermShift;
                rb.r32.push_back(a);
                if (rb.want64) {
                    koma::Rec64 b{};
                    b.type = koma::REC_PREC;
                    for (int d = 0; d < 3; ++d) {
                        b.a[d] = c.K[d];
                        b.a[4 + d] = c.K1[d];
                    }
                    b.a[3] = c.tau;
                    rb.r64.push_back(b);
                }
                if (rb.wantM) {
                    koma::RecM m = RecordBuilder::extend(a);
                    for (int d = 0; d < 3; ++d) split(c.K1[d], &m.a[8 + 2 * d], &m.a[9 + 2 * d]);
                    m.count = a.count | (RecordBuilder::k1_bits(m, 8) << koma::kTermShift);
                    rb.rm.push_back(m);
                }
                ++rb.n_mat;
            }
            koma::Rec32 a{};
            a.type = koma::REC_RF;
            const double s = kGammaBar * dt[n];  // turns per tesla
            // FP32 record: half-angle vector pi s B (radians); FP64: s B (turns)
            for (int d = 0; d < 3; ++d) a.a[d] = static_cast<float>(kPi * s * gm[d]);
            const double bx = s * b1_re[n], by = s * b1_im[n];
            a.a[3] = static_cast<float>(kPi * bx);
            a.a[4] = static_cast<float>(kPi * by);
            // |theta_xy|^2 of the FP32 values; kept above zero so the general
            // path's rsqrt stays finite for a vanishing field
            a.a[5] = std::max(a.a[3] * a.a[3] + a.a[4] * a.a[4], std::numeric_limits<float>::min());
            a.a[6] = static_cast<float>(dt[n]);
            rb.r32.push_back(a);
            const double t_mid = t + 0.5 * dt[n];
            if (rb.want64) {
                koma::Rec64 b{};
                b.type = koma::REC_RF;
                for (int d = 0; d < 3; ++d) b.a[d] = s * gm[d];
                b.a[3] = bx;
                b.a[4] = by;
                b.a[5] = dt[n];
                b.a[6] = t_mid;
                rb.r64.push_back(b);
            }
            if (rb.wantM) {
                koma::RecM m = RecordBuilder::extend(a);
                m.a[13] = static_cast<float>(t_mid);
                rb.rm.push_back(m);
            }
            for (int d = 0; d < 3; ++d) c.K[d] = c.K1[d] = 0.0;
            c.tau = 0.0;
        } else {
            ++c.n_precess;
            const double g0[3] = {gx[n], gy[n], gz[n]}, g1[3] = {gx[n + 1], gy[n + 1], gz[n + 1]};
            for (int d = 0; d < 3; ++d) {
                c.K[d] += kGammaBar * dt[n] * gm[d];
                // integral of a linear G times s over [t, t_next]
                c.K1[d] += kGammaBar * dt[n] / 6.0 * (g0[d] * (2.0 * t + t_next) + g1[d] * (t + 2.0 * t_next));
            }
            c.tau += dt[n];
        }
        t = t_next;
        if (adc[n + 1]) rb.sample(c.K, c.K1, c.tau);
    }
}

// Builders of the parallel chunks, kept between builds (their vectors stay
// allocated: the next build writes warm memory).
std::mutex g_builders_mu;
std::vector<RecordBuilder*> g_builders;

RecordBuilder* builder_acquire() {
    {
        std::lock_guard<std::mutex> lk(g_builders_mu);
        if (!g_builders.empty()) {
            RecordBuilder* b = g_builders.back();
            g_builders.pop_back();
            return b;
        }
    }
    return new RecordBuilder();
}

void builder_release(RecordBuilder* b) {
    std::lock_guard<std::mutex> lk(g_builders_mu);
    g_builders.push_back(b);
}

// Workers for k chunks (the host pool's size, at most k).
int n_workers_for(int k) {
    const unsigned hw = std::max(1u, std::min(std::thread::hardware_concurrency(), 16u));
    return std::max(1, std::min(k, static_cast<int>(hw)));
}

// run(w) for w in [0, k) on the host pool, or one after another on the
// calling thread when the pool is busy.
void run_tasks(int k, const std::function<void(int)>& run) {
    if (k <= 1 || !t_host_parallel) {
        for (int w = 0; w < k; ++w) run(w);
        return;
    }
    if (k <= 1) {
        run(0);
        return;
    }
    if (HostPool::get().try_run(k, run)) return;
    for (int w = 0; w < k; ++w) run(w);  // the pool is busy: serial (see parallel_for)
}

// The FP32 records of a parallel build left in the chunk builders: the
// FP32-only upload copies them, in parallel, straight to their places in its
// staging buffer instead of concatenating them into one vector first.
struct PendingChunks {
    struct Part {
        int w;                    // builder
        size_t r0, r1, dst;       // its records [r0, r1) go to dst
    };
    std::vector<RecordBuilder*> wb;
    std::vector<Part> parts;
    size_t n32 = 0;
    bool active() const { return !wb.empty(); }
    void gather(koma::Rec32* dst) const {
        const int k = n_workers_for(static_cast<int>(parts.size()));
        run_tasks(k, [&](int t) {
            for (size_t i = static_cast<size_t>(t); i < parts.size(); i += static_cast<size_t>(k)) {
                const Part& q = parts[i];
                if (q.r1 > q.r0)
                    std::memcpy(dst + q.dst, wb[q.w]->r32.data() + q.r0, (q.r1 - q.r0) * sizeof(koma::Rec32));
            }
        });
    }
    void release() {
        for (RecordBuilder* b : wb) builder_release(b);
        wb.clear();
        parts.clear();
    }
    ~PendingChunks() { release(); }
};

// Validation + preprocessing shared by koma_sequence_upload and
// koma_sequence_plan. `err` receives the message on failure. With `pend`
// (FP32 stream only: neither FP64 nor motion records wanted), a build in
// parallel chunks leaves its records in the chunk builders (rb.r32 stays
// empty) for the caller to gather.
koma_status build_records(int64_t n_steps, const double* dt, const double* gx, const double* gy,
                          const double* gz, const double* b1_re, const double* b1_im, const uint8_t* adc,
                          RecordBuilder& rb, koma_sequence_info& info, std::string& err,
                          PendingChunks* pend = nullptr) {
    char buf[256];
    auto bad = [&](const char* fmt, long long i, double v) {
        snprintf(buf, sizeof(buf), fmt, i, v);
        err = buf;
        return KOMA_E_INVALID;
    };
    if (n_steps < 0) return bad("sequence: n_steps = %lld < 0%.0g", n_steps, 0.0);
    if (!gx || !gy || !gz || !adc || (n_steps > 0 && (!dt || !b1_re || !b1_im)))
        return bad("sequence: NULL array (n_steps %lld)%.0g", n_steps, 0.0);
    // long sequences: a parallel pass finds whether anything is invalid, and
    // only then do the serial loops below look for the first offending index
    bool check_serially = true;
    if (n_steps >= 65536) {
        const int k = n_workers_for(16);
        std::vector<uint8_t> bad_in(static_cast<size_t>(k), 0);
        run_tasks(k, [&](int w) {
            const int64_t lo = n_steps * w / k, hi = w + 1 == k ? n_steps + 1 : n_steps * (w + 1) / k;
            bool b = false;
            for (int64_t i = lo; i < hi; ++i) {
                b |= !std::isfinite(gx[i]) || !std::isfinite(gy[i]) || !std::isfinite(gz[i]) || adc[i] > 1;
                if (i < n_steps)
                    b |= !std::isfinite(dt[i]) || !(dt[i] > 0) || !std::isfinite(b1_re[i]) || !std::isfinite(b1_im[i]);
            }
            bad_in[w] = b;
        });
        check_serially = std::find(bad_in.begin(), bad_in.end(), 1) != bad_in.end();
    }
    if (check_serially) {
        for (int64_t i = 0; i <= n_steps; ++i) {
            if (!std::isfinite(gx[i]) || !std::isfinite(gy[i]) || !std::isfinite(gz[i]))
                return bad("sequence: non-finite gradient at time point %lld%.0g", i, 0.0);
            if (adc[i] > 1) return bad("sequence: adc[%lld] = %g (must be 0 or 1)", i, adc[i]);
        }
        for (int64_t n = 0; n < n_steps; ++n) {
            if (!std::isfinite(dt[n]) || !(dt[n] > 0))
                return bad("sequence: dt[%lld] = %g (must be finite and > 0)", n, dt[n]);
            if (!std::isfinite(b1_re[n]) || !std::isfinite(b1_im[n]))
                return bad("sequence: non-finite B1 at step %lld%.0g", n, 0.0);
        }
    }
    info = koma_sequence_info{};
    info.n_steps = n_steps;
    // Long sequences are built in parallel chunks. A chunk starts at a step
    // a that is not RF, follows the last step of an RF run, and whose time
    // point a carries no sample:
    // there the moments since t_ref are zero and no ADC run is open, so the
    // chunk needs only the absolute time and the number of samples before
    // it, which one serial pass gives (t summed in the same order as the
    // serial build: the records are bitwise the same).
    std::vector<int64_t> cut{0};
    std::vector<double> t_at{0.0};
    std::vector<int64_t> adc_at{0};
    const int64_t kChunkSteps = 2048;
    if (n_steps >= 2 * kChunkSteps) {
        double t = 0.0;
        int64_t na = adc[0];
        int64_t next = kChunkSteps;
        for (int64_t n = 0; n < n_steps; ++n) {
            // step n - 1 ends an RF run (step n is not RF), time point n has no sample
            if (n >= next && n > 0 && (b1_re[n - 1] != 0.0 || b1_im[n - 1] != 0.0) && b1_re[n] == 0.0 &&
                b1_im[n] == 0.0 && !adc[n]) {
                cut.push_back(n);
                t_at.push_back(t);
                adc_at.push_back(na);
                next = n + kChunkSteps;
            }
            t = t + dt[n];
            na += adc[n + 1];
        }
    }
    cut.push_back(n_steps);
    const int n_chunks = static_cast<int>(cut.size()) - 1;
    if (n_chunks == 1) {
        BuildCounts c;
        if (adc[0]) rb.sample(c.K, c.K1, c.tau);
        build_steps(0, n_steps, 0.0, dt, gx, gy, gz, b1_re, b1_im, adc, rb, c);
        rb.close_run();
        rb.mark_rf_runs();
        info.n_rf = c.n_rf;
        info.n_precess = c.n_precess;
    } else {
        // worker w builds chunks w, w + k, ... into a builder it keeps (warm
        // memory), one after another; the chunks are then concatenated in
        // order. No RF run crosses a cut, and a chunk never starts with an RF
        // record (its first step is not RF and has dt > 0).
        const int k = n_workers_for(n_chunks);
        struct Range {
            size_t r32[2], r64[2], rm[2];
            int64_t n_adc_end;
        };
        std::vector<Range> rng(static_cast<size_t>(n_chunks));
        std::vector<BuildCounts> cnt(static_cast<size_t>(n_chunks));
        std::vector<RecordBuilder*> wb(static_cast<size_t>(k), nullptr);
        for (int w = 0; w < k; ++w) wb[w] = builder_acquire();
        const std::function<void(int)> run = [&](int w) {
            RecordBuilder& tl = *wb[w];
            tl.reset(rb.want64, rb.wantM);
            for (int i = w; i < n_chunks; i += k) {
                Range& R = rng[i];
                R.r32[0] = tl.r32.size();
                R.r64[0] = tl.r64.size();
                R.rm[0] = tl.rm.size();
                tl.n_adc = adc_at[i];
                BuildCounts c;  // local: the chunks' counters share cache lines
                if (i == 0 && adc[0]) tl.sample(c.K, c.K1, c.tau);
                build_steps(cut[i], cut[i + 1], t_at[i], dt, gx, gy, gz, b1_re, b1_im, adc, tl, c);
                cnt[i] = c;
                tl.close_run();
                R.r32[1] = tl.r32.size();
                R.r64[1] = tl.r64.size();
                R.rm[1] = tl.rm.size();
                R.n_adc_end = tl.n_adc;
            }
            tl.mark_rf_runs();
        };
        run_tasks(k, run);
        size_t n32 = 0, n64 = 0, nm = 0;
        for (int w = 0; w < k; ++w) {
            n32 += wb[w]->r32.size();
            n64 += wb[w]->r64.size();
            nm += wb[w]->rm.size();
            rb.n_runs += wb[w]->n_runs;
            rb.n_mat += wb[w]->n_mat;
        }
        if (pend && !rb.want64 && !rb.wantM) {
            // the caller gathers: chunk i's records go after those of chunks < i
            pend->release();
            size_t at = 0;
            for (int i = 0; i < n_chunks; ++i) {
                const Range& R = rng[i];
                pend->parts.push_back({i % k, R.r32[0], R.r32[1], at});
                at += R.r32[1] - R.r32[0];
                info.n_rf += cnt[i].n_rf;
                info.n_precess += cnt[i].n_precess;
            }
            pend->wb = wb;
            pend->n32 = at;
            rb.n_adc = rng[n_chunks - 1].n_adc_end;
            info.n_adc = rb.n_adc;
            info.n_records = static_cast<int64_t>(at);
            info.n_adc_runs = rb.n_runs;
            info.n_materialize = rb.n_mat;
            return KOMA_OK;
        }
        rb.r32.reserve(n32);
        if (rb.want64) rb.r64.reserve(n64);
        if (rb.wantM) rb.rm.reserve(nm);
        for (int i = 0; i < n_chunks; ++i) {
            const RecordBuilder& b = *wb[i % k];
            const Range& R = rng[i];
            rb.r32.insert(rb.r32.end(), b.r32.begin() + R.r32[0], b.r32.begin() + R.r32[1]);
            if (rb.want64) rb.r64.insert(rb.r64.end(), b.r64.begin() + R.r64[0], b.r64.begin() + R.r64[1]);
            if (rb.wantM) rb.rm.insert(rb.rm.end(), b.rm.begin() + R.rm[0], b.rm.begin() + R.rm[1]);
            info.n_rf += cnt[i].n_rf;
            info.n_precess += cnt[i].n_precess;
        }
        rb.n_adc = rng[n_chunks - 1].n_adc_end;
        for (int w = 0; w < k; ++w) builder_release(wb[w]);
    }
    info.n_adc = rb.n_adc;
    info.n_records = static_cast<int64_t>(rb.r32.size());
    info.n_adc_runs = rb.n_runs;
    info.n_materialize = rb.n_mat;
    return KOMA_OK;
}

}  // namespace

// Matrix-form readout plan. ADC records of at least two samples are bucketed
// by their rotator (dK, dtau as FP32 bit patterns); a bucket of at least
// kMmaMinRuns runs and kMmaMinSamples samples is taken by the tensor-core
// readout: its records get kMmaFlag and its runs form groups of up to
// kMmaRuns in record order. Blocks (stretches between RF and PREC records,
// where the state is constant) holding taken runs get one snapshot row each,
// in record order; the first taken record of such a block also gets
// kMmaSnapFlag (the Bloch kernel stores the snapshot there).
struct MmaPlan {
    std::vector<koma::MmaGroup> groups;
    std::vector<koma::MmaRun> runs;
    std::vector<uint8_t> from;  // [n_adc]: 1 = sample taken by the matrix form
    int64_t n_samples = 0;
    int64_t n_snaps = 0;
};

// Length of the run of RF records that starts at record i: the builder
// stores it in the run's first record (RecordBuilder::mark_rf_runs), so the
// plans step over a pulse's records instead of visiting each; a run without
// it is counted.
size_t rf_run_len(koma::RecSpan r32, size_t i) {
    const int32_t c = r32[i].count;
    if (c > 0 && i + static_cast<size_t>(c) <= r32.size()) return static_cast<size_t>(c);
    size_t j = i;
    while (j < r32.size() && r32[j].type == koma::REC_RF) ++j;
    return j - i;
}

void plan_mma(koma::RecSpan r32, int64_t n_adc, MmaPlan& P) {
    std::map<std::array<uint32_t, 4>, std::vector<size_t>> buckets;
    for (size_t i = 0; i < r32.size(); ++i) {
        const koma::Rec32& R = r32[i];
        if (R.type == koma::REC_RF) {
            i += rf_run_len(r32, i) - 1;
            continue;
        }
        if (R.type != koma::REC_ADC || (R.count & koma::kCountMask) < 2) continue;
        std::array<uint32_t, 4> key;
        std::memcpy(key.data(), &R.a[8], sizeof(key));
        buckets[key].push_back(i);
    }
    std::vector<char> taken(r32.size(), 0);
    std::vector<const std::vector<size_t>*> chosen;
    for (const auto& kv : buckets) {
        int64_t samples = 0;
        for (size_t i : kv.second) samples += r32[i].count & koma::kCountMask;
        if (static_cast<int64_t>(kv.second.size()) >= koma::kMmaMinRuns && samples >= koma::kMmaMinSamples) {
            chosen.push_back(&kv.second);
            for (size_t i : kv.second) taken[i] = 1;
        }
    }
    if (chosen.empty()) return;
    // snapshot rows: one per block holding taken runs
    std::vector<int32_t> snap(r32.size(), -1);
    int32_t next = 0;
    bool block_has = false;
    for (size_t i = 0; i < r32.size(); ++i) {
        koma::Rec32& R = r32[i];
        if (R.type != koma::REC_ADC) {
            block_has = false;  // RF or PREC: the state changes, a new block begins
            if (R.type == koma::REC_RF) i += rf_run_len(r32, i) - 1;
            continue;
        }
        if (!taken[i]) continue;
        R.count |= koma::kMmaFlag;
        if (!block_has) {
            R.count |= koma::kMmaSnapFlag;
            ++next;
            block_has = true;
        }
        snap[i] = next - 1;
    }
    P.n_snaps = next;
    P.from.assign(static_cast<size_t>(n_adc), 0);
    for (const std::vector<size_t>* v : chosen) {
        for (size_t g0 = 0; g0 < v->size(); g0 += koma::kMmaRuns) {
            const size_t g1 = std::min(v->size(), g0 + static_cast<size_t>(koma::kMmaRuns));
            koma::MmaGroup G{};
            const koma::Rec32& H = r32[(*v)[g0]];
            G.dk[0] = H.a[8];
            G.dk[1] = H.a[9];
            G.dk[2] = H.a[10];
            G.dtau = H.a[11];
            G.run0 = static_cast<int32_t>(P.runs.size());
            G.n_runs = static_cast<int32_t>(g1 - g0);
            G.one_snap = 1;
            for (size_t q = g0; q < g1; ++q) {
                const koma::Rec32& R = r32[(*v)[q]];
                koma::MmaRun run{};
                run.k0 = R.k0;
                run.len = R.count & koma::kCountMask;
                run.snap = snap[(*v)[q]];
                for (int d = 0; d < 3; ++d) {
                    run.kh[d] = R.a[2 * d];
                    run.kl[d] = R.a[2 * d + 1];
                }
                run.th = R.a[6];
                run.tl = R.a[7];
                G.max_len = std::max(G.max_len, run.len);
                if (run.snap != snap[(*v)[g0]]) G.one_snap = 0;
                P.n_samples += run.len;
                P.runs.push_back(run);
                std::fill(P.from.begin() + run.k0, P.from.begin() + run.k0 + run.len, 1);
            }
            P.groups.push_back(G);
        }
    }
}

// Repeated RF pulses: runs of consecutive RF records whose 64-byte records
// are bitwise equal (the same pulse under the same gradient, so the same
// per-spin map) are grouped; a group of at least kRfMapMinRuns runs of at
// least kRfMapMinLen steps gets a map slot (at most kMaxRfMaps, the ones
// saving the most steps first), and the header record of each of its runs
// gets k0 = 1 + slot.
struct RfMapPlan {
    std::vector<koma::RfMapPulse> pulses;
    int64_t runs = 0, steps = 0, pulse_steps = 0;
};

void plan_rf_maps(koma::RecSpan r32, RfMapPlan& P) {
    struct Run {
        size_t begin, len;
    };
    // the maximal runs of RF records, stepped over by their stored lengths
    const size_t n_rec = r32.size();
    std::vector<Run> runs;
    for (size_t i = 0; i < n_rec;) {
        if (r32[i].type != koma::REC_RF) {
            ++i;
            continue;
        }
        const size_t len = rf_run_len(r32, i);
        runs.push_back({i, len});
        i += len;
    }
    const bool par = n_rec >= 16384;
    auto same = [&](const Run& a, const Run& b) {
        return a.len == b.len && std::memcmp(&r32[a.begin], &r32[b.begin], a.len * sizeof(koma::Rec32)) == 0;
    };
    // a multiplicative hash of the run's 8-byte words buckets the candidates;
    // equality is checked byte for byte
    // the runs' hashes, in parallel for long sequences (runs are independent)
    std::vector<uint64_t> hash(runs.size(), 0);
    auto hash_runs = [&](size_t q0, size_t q1) {
        for (size_t q = q0; q < q1; ++q) {
            if (runs[q].len < static_cast<size_t>(koma::kRfMapMinLen)) continue;
            uint64_t h = 1469598103934665603ull;
            const unsigned char* b = reinterpret_cast<const unsigned char*>(&r32[runs[q].begin]);
            for (size_t k = 0; k < runs[q].len * sizeof(koma::Rec32); k += 8) {  // 64-byte records: whole words
                uint64_t w;
                std::memcpy(&w, b + k, 8);
                h = (h ^ w) * 1099511628211ull;
                h ^= h >> 29;
            }
            hash[q] = h;
        }
    };
    const bool par_runs = par && runs.size() >= 16;
    if (par_runs) {
        const int k = n_workers_for(static_cast<int>(std::min<size_t>(runs.size(), 64)));
        run_tasks(k, [&](int w) { hash_runs(runs.size() * w / k, runs.size() * (w + 1) / k); });
    } else {
        hash_runs(0, runs.size());
    }
    // equality with the first run of the same hash and length, checked byte
    // for byte (in parallel for long streams); a run that differs from it (a
    // hash collision) is placed by comparing it with every class of its bucket
    std::map<std::pair<uint64_t, size_t>, size_t> first;
    std::vector<size_t> rep(runs.size(), SIZE_MAX);
    for (size_t q = 0; q < runs.size(); ++q) {
        if (runs[q].len < static_cast<size_t>(koma::kRfMapMinLen)) continue;
        rep[q] = first.emplace(std::make_pair(hash[q], runs[q].len), q).first->second;
    }
    std::vector<uint8_t> eq(runs.size(), 0);
    auto check = [&](size_t q0, size_t q1) {
        for (size_t q = q0; q < q1; ++q)
            if (rep[q] != SIZE_MAX) eq[q] = rep[q] == q || same(runs[rep[q]], runs[q]);
    };
    if (par_runs) {
        const int k = n_workers_for(static_cast<int>(std::min<size_t>(runs.size(), 64)));
        run_tasks(k, [&](int w) { check(runs.size() * w / k, runs.size() * (w + 1) / k); });
    } else {
        check(0, runs.size());
    }
    std::map<std::pair<uint64_t, size_t>, std::vector<std::vector<size_t>>> buckets;
    for (size_t q = 0; q < runs.size(); ++q) {
        if (rep[q] == SIZE_MAX) continue;
        auto& classes = buckets[{hash[q], runs[q].len}];
        if (eq[q] && !classes.empty() && classes[0][0] == rep[q]) {
            classes[0].push_back(q);  // equal to the bucket's first run: its class
            continue;
        }
        bool placed = false;
        for (size_t ci = eq[q] ? 0 : 1; ci < classes.size() && !placed; ++ci) {
            if (same(runs[classes[ci][0]], runs[q])) {
                classes[ci].push_back(q);
                placed = true;
            }
        }
        if (!placed) classes.push_back({q});
    }
    std::vector<const std::vector<size_t>*> cand;
    for (const auto& kv : buckets)
        for (const auto& c : kv.second)
            if (c.size() >= static_cast<size_t>(koma::kRfMapMinRuns)) cand.push_back(&c);
    // most stepped RF steps saved first; ties by first occurrence
    std::sort(cand.begin(), cand.end(), [&](const std::vector<size_t>* a, const std::vector<size_t>* b) {
        const size_t sa = (a->size() - 1) * runs[(*a)[0]].len, sb = (b->size() - 1) * runs[(*b)[0]].len;
        return sa != sb ? sa > sb : (*a)[0] < (*b)[0];
    });
    if (cand.size() > static_cast<size_t>(koma::kMaxRfMaps)) cand.resize(koma::kMaxRfMaps);
    for (size_t slot = 0; slot < cand.size(); ++slot) {
        const Run& first = runs[(*cand[slot])[0]];
        koma::RfMapPulse p{};
        p.rec_begin = static_cast<int64_t>(first.begin);
        p.len = static_cast<int32_t>(first.len);
        P.pulses.push_back(p);
        P.pulse_steps += static_cast<int64_t>(first.len);
        for (size_t q : *cand[slot]) {
            r32[runs[q].begin].k0 = static_cast<int64_t>(slot) + 1;
            P.runs += 1;
            P.steps += static_cast<int64_t>(runs[q].len);
        }
    }
}

namespace {
bool z_dictionary_stream(koma::RecSpan r32);
double build_z_stream(koma::RecSpan r32, std::vector<koma::Rec32>& out);
}  // namespace

extern "C" koma_status koma_sequence_plan(int64_t n_steps, const double* dt, const double* gx, const double* gy,
                                          const double* gz, const double* b1_re, const double* b1_im,
                                          const uint8_t* adc, koma_sequence_info* info, double* rec_out,
                                          int64_t rec_capacity) {
    if (!info) return KOMA_E_INVALID;
    RecordBuilder rb;
    std::string err;
    koma_status st = build_records(n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, rb, *info, err);
    if (st != KOMA_OK) return st;
    MmaPlan mp;
    plan_mma(rb.r32, info->n_adc, mp);
    info->n_mma_groups = static_cast<int64_t>(mp.groups.size());
    info->n_mma_runs = static_cast<int64_t>(mp.runs.size());
    info->n_mma_samples = mp.n_samples;
    RfMapPlan fp;
    plan_rf_maps(rb.r32, fp);
    info->n_rf_maps = static_cast<int64_t>(fp.pulses.size());
    info->n_rf_map_runs = fp.runs;
    info->n_rf_map_steps = fp.steps;
    info->n_rf_map_pulse_steps = fp.pulse_steps;
    info->z_dict = z_dictionary_stream(rb.r32) ? 1 : 0;
    if (info->z_dict) {
        std::vector<koma::Rec32> rz;
        info->z_kmax = build_z_stream(rb.r32, rz);
    }
    if (rec_out) {
        if (rec_capacity < info->n_records) return KOMA_E_INVALID;
        for (int64_t r = 0; r < info->n_records; ++r) {
            const koma::Rec64& q = rb.r64[static_cast<size_t>(r)];
            double* o = rec_out + 17 * r;
            o[0] = q.type;
            o[1] = q.count;
            o[2] = static_cast<double>(q.k0);
            for (int i = 0; i < 14; ++i) o[3 + i] = q.a[i];
        }
    }
    return KOMA_OK;
}

namespace {

// Sequence upload. The records are built by a builder the calling thread
// keeps (its vectors stay warm from one upload to the next), the device
// block [Rec32 | Rec64 | RecM | MmaGroup | MmaRun | sample map | RfMapPulse |
// compacted Rec32] (each part 16-byte aligned) is assembled in the
// context's pinned staging buffer and copied by DMA. need64 / needM: build
// and upload the FP64 and the motion record streams (koma_sequence_upload
// builds every stream; callers that know the precision, and that the
// phantom is static, build the FP32 stream only).
// The record stream's side of K3z's condition: no RF step has a z gradient
// (its rotation is the same for spins that differ only in z) and no ADC
// record holds more than one sample.
bool z_dictionary_stream(koma::RecSpan r32) {
    for (const koma::Rec32& R : r32) {
        if (R.type == koma::REC_RF && (R.a[2] != 0.f || (R.count > 0 && R.a[10] != 0.f))) return false;
        if (R.type == koma::REC_ADC && (R.count & koma::kCountMask) > 1) return false;
    }
    return true;
}

// K3z's record stream: a copy of the FP32 stream in which
// * an RF record's a[0..8] hold the step's rotation as a 3x3 matrix (row
//   major) and a[9] its dt. The rotation is that of the uniform RF path:
//   the quaternion (ch, ux, uy, 0) = (cos h, -sin h / h (bx, by), 0) of half
//   angle h = sqrt(b2) applied as v + c2 (ch u x v + u x (u x v)) with the
//   first-order renormalisation c2 = 4 - 2 |q|^2, i.e. the matrix
//   I + c2 (ch [u]x + [u]x^2), evaluated in FP64 from the record's FP32
//   fields and rounded once per entry;
// * a PREC/ADC record's a[8] holds -2 pi Kz (Kz = hi + lo, FP64, rounded once),
//   the phase per metre of z when the phantom's extent keeps |z Kz| small.
// Everything else is copied. Returns max |Kz| over the records with a z term.
double build_z_stream(koma::RecSpan r32, std::vector<koma::Rec32>& out) {
    out.assign(r32.begin(), r32.end());
    double kmax = 0.0;
    for (koma::Rec32& R : out) {
        if (R.type == koma::REC_RF) {
            const double bx = R.a[3], by = R.a[4], b2 = R.a[5], dt = R.a[6];
            double ch = 1.0, f = -1.0;
            if (b2 > 0.0) {
                const double h = std::sqrt(b2);
                ch = std::cos(h);
                f = -std::sin(h) / h;
            }
            const double ux = bx * f, uy = by * f, s = ux * ux + uy * uy;
            const double c2 = 4.0 - 2.0 * (ch * ch + s);
            const double m[9] = {1.0 - c2 * uy * uy, c2 * ux * uy,       c2 * ch * uy,
                                 c2 * ux * uy,       1.0 - c2 * ux * ux, -c2 * ch * ux,
                                 -c2 * ch * uy,      c2 * ch * ux,       1.0 - c2 * s};
            for (int k = 0; k < 9; ++k) R.a[k] = static_cast<float>(m[k]);
            R.a[9] = static_cast<float>(dt);
        } else if (R.type == koma::REC_PREC || R.type == koma::REC_ADC) {
            const double kz = static_cast<double>(R.a[4]) + static_cast<double>(R.a[5]);
            R.a[8] = static_cast<float>(-2.0 * kPi * kz);
            if ((R.count >> koma::kTermShift) & 4) kmax = std::max(kmax, std::fabs(kz));
        }
    }
    return kmax;
}

// The context's pinned staging buffer holds at least `need` bytes; when it
// grows, its first `keep` bytes move to the new buffer (no copy is in flight:
// uploads from it are synchronous).
koma_status stage_reserve(koma_ctx* ctx, size_t need, size_t keep) {
    if (need <= ctx->h_stage_bytes) return KOMA_OK;
    const size_t want = (need + need / 4 + (size_t{1} << 20) - 1) / (size_t{1} << 20) * (size_t{1} << 20);
    char* h = nullptr;
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&h), want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sequence_upload: staging buffer");
    }
    if (keep && ctx->h_stage) std::memcpy(h, ctx->h_stage, std::min(keep, ctx->h_stage_bytes));
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = h;
    ctx->h_stage_bytes = want;
    return KOMA_OK;
}

koma_status sequence_upload_impl(koma_ctx* ctx, int64_t n_steps, const double* dt, const double* gx,
                                 const double* gy, const double* gz, const double* b1_re, const double* b1_im,
                                 const uint8_t* adc, bool need64, bool needM, koma_sequence** out) {
    if (!ctx) return KOMA_E_INVALID;
    if (!out) return fail(ctx, KOMA_E_INVALID, "sequence_upload: out is NULL");
    *out = nullptr;
    static thread_local RecordBuilder rb;
    rb.reset(need64, needM);
    koma_sequence_info info{};
    PendingChunks pend;
    {
        std::string err;
        koma_status st = build_records(n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, rb, info, err, &pend);
        if (st != KOMA_OK) return fail(ctx, st, "%s", err.c_str());
    }
    // the FP32 records: the builder's vector, or (a parallel build of the FP32
    // stream alone) gathered straight into the staging buffer, where the plans
    // below mark them in place
    const bool gathered = pend.active();
    koma::RecSpan recs(rb.r32);
    if (gathered) {
        const koma_status st = stage_reserve(ctx, pend.n32 * sizeof(koma::Rec32), 0);
        if (st != KOMA_OK) return st;
        pend.gather(reinterpret_cast<koma::Rec32*>(ctx->h_stage));
        recs = koma::RecSpan(reinterpret_cast<koma::Rec32*>(ctx->h_stage), pend.n32);
        pend.release();
    }
    koma_sequence* seq = new (std::nothrow) koma_sequence();
    if (!seq) return fail(ctx, KOMA_E_NOMEM, "sequence_upload: host allocation");
    seq->ctx = ctx;
    seq->info = info;
    seq->z_dict = z_dictionary_stream(recs);
    std::vector<koma::Rec32> rz;
    if (seq->z_dict) seq->z_kmax = build_z_stream(recs, rz);
    seq->info.z_dict = seq->z_dict ? 1 : 0;
    seq->info.z_kmax = seq->z_kmax;
    MmaPlan mp;
    plan_mma(recs, info.n_adc, mp);
    seq->info.n_mma_groups = static_cast<int64_t>(mp.groups.size());
    seq->info.n_mma_runs = static_cast<int64_t>(mp.runs.size());
    seq->info.n_mma_samples = mp.n_samples;
    RfMapPlan fp;
    plan_rf_maps(recs, fp);
    seq->info.n_rf_maps = static_cast<int64_t>(fp.pulses.size());
    seq->info.n_rf_map_runs = fp.runs;
    seq->info.n_rf_map_steps = fp.steps;
    seq->info.n_rf_map_pulse_steps = fp.pulse_steps;
    // the compacted stream's length (the stream itself is written into the block)
    const size_t n_rc = fp.pulses.empty() ? 0 : koma::compact_records32_into(recs.p, recs.n, nullptr);
    DeviceGuard g(ctx->device);
    auto up16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t b32 = recs.size() * sizeof(koma::Rec32), b64 = rb.r64.size() * sizeof(koma::Rec64),
                 bm = rb.rm.size() * sizeof(koma::RecM), bg = mp.groups.size() * sizeof(koma::MmaGroup),
                 br = mp.runs.size() * sizeof(koma::MmaRun), bf = up16(mp.from.size()),
                 bp = fp.pulses.size() * sizeof(koma::RfMapPulse), bc = n_rc * sizeof(koma::Rec32),
                 bz = rz.size() * sizeof(koma::Rec32);
    const size_t total = b32 + b64 + bm + bg + br + bf + bp + bc + bz;
    koma_status st = dev_alloc(ctx, reinterpret_cast<void**>(&seq->r32), total, "sequence_upload");
    // the whole block in the staging buffer (keeping gathered records)
    if (st == KOMA_OK) st = stage_reserve(ctx, total, gathered ? b32 : 0);
    if (gathered) recs.p = reinterpret_cast<koma::Rec32*>(ctx->h_stage);
    if (st == KOMA_OK && b32) {
        char* base = reinterpret_cast<char*>(seq->r32);
        char* h = ctx->h_stage;
        if (b64) seq->r64 = reinterpret_cast<koma::Rec64*>(base + b32);
        if (bm) seq->rm = reinterpret_cast<koma::RecM*>(base + b32 + b64);
        size_t off = b32 + b64 + bm;
        if (!mp.groups.empty()) {
            seq->d_mma_groups = reinterpret_cast<koma::MmaGroup*>(base + off);
            seq->d_mma_runs = reinterpret_cast<koma::MmaRun*>(base + off + bg);
            seq->d_from_mma = reinterpret_cast<uint8_t*>(base + off + bg + br);
            seq->n_mma_groups = static_cast<int32_t>(mp.groups.size());
            seq->n_mma_runs = static_cast<int64_t>(mp.runs.size());
            seq->n_mma_snaps = mp.n_snaps;
        }
        if (!gathered) std::memcpy(h, rb.r32.data(), b32);
        if (b64) std::memcpy(h + b32, rb.r64.data(), b64);
        if (bm) std::memcpy(h + b32 + b64, rb.rm.data(), bm);
        if (bg) std::memcpy(h + off, mp.groups.data(), bg);
        if (br) std::memcpy(h + off + bg, mp.runs.data(), br);
        if (bf) {
            std::memcpy(h + off + bg + br, mp.from.data(), mp.from.size());
            std::memset(h + off + bg + br + mp.from.size(), 0, bf - mp.from.size());
        }
        off += bg + br + bf;
        if (bp) {
            seq->d_rf_pulses = reinterpret_cast<koma::RfMapPulse*>(base + off);
            seq->n_rf_maps = static_cast<int32_t>(fp.pulses.size());
            seq->r32c = reinterpret_cast<koma::Rec32*>(base + off + bp);
            seq->n_rec_c = static_cast<int64_t>(n_rc);
            std::memcpy(h + off, fp.pulses.data(), bp);
            koma::compact_records32_into(recs.p, recs.n, reinterpret_cast<koma::Rec32*>(h + off + bp));
        }
        off += bp + bc;
        if (bz) {
            seq->r32z = reinterpret_cast<koma::Rec32*>(base + off);
            std::memcpy(h + off, rz.data(), bz);
        }
        cudaError_t e = h2d_sync(ctx, seq->r32, h, total);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "sequence_upload: copy");
    }
    if (st != KOMA_OK) {
        dev_free(ctx, seq->r32, total);
        delete seq;
        return st;
    }
    seq->bytes = total;
    ctx->live_objects++;
    *out = seq;
    return KOMA_OK;
}

}  // namespace

extern "C" koma_status koma_sequence_upload(koma_ctx* ctx, int64_t n_steps, const double* dt, const double* gx,
                                            const double* gy, const double* gz, const double* b1_re,
                                            const double* b1_im, const uint8_t* adc, koma_sequence** out) {
    NvtxRange nvtx_("koma_sequence_upload");
    return sequence_upload_impl(ctx, n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, true, true, out);
}

extern "C" int64_t koma_sequence_n_adc(const koma_sequence* seq) { return seq ? seq->info.n_adc : -1; }
extern "C" int64_t koma_sequence_n_steps(const koma_sequence* seq) { return seq ? seq->info.n_steps : -1; }

extern "C" koma_status koma_sequence_get_info(const koma_sequence* seq, koma_sequence_info* info) {
    if (!seq || !info) return KOMA_E_INVALID;
    *info = seq->info;
    return KOMA_OK;
}

extern "C" koma_status koma_sequence_free(koma_sequence* seq) {
    if (!seq) return KOMA_OK;
    koma_ctx* ctx = seq->ctx;
    DeviceGuard g(ctx->device);
    dev_free(ctx, seq->r32, seq->bytes);
    ctx->live_objects--;
    delete seq;
    return KOMA_OK;
}

// ---------------------------------------------------------------------------
// simulate
// ---------------------------------------------------------------------------
namespace {

// Phantom extents as FP32 upper bounds (the kernels bound each RF step's
// rotation with them).
void phantom_ext(const koma_phantom* ph, float (&ext)[4], int* used) {
    *used = 0;
    for (int d = 0; d < 4; ++d) {
        ext[d] = static_cast<float>(ph->max_abs[d] * (1.0 + 1e-6));
        if (ph->max_abs[d] > 0) *used |= 1 << d;
    }
}

// Velocity block, extents and used bits of a moving phantom.
void motion_args(const koma_phantom* ph, koma::BlochArgs& A) {
    A.pv32 = ph->pv32;
    A.pv64 = ph->pv64;
    for (int d = 0; d < 3; ++d) {
        A.vext[d] = static_cast<float>(ph->max_v[d] * (1.0 + 1e-6));
        if (ph->max_v[d] > 0) A.used |= 1 << (4 + d);
    }
}

// Split every group into work items of 32 S spins (one warp each, every lane
// slot full) plus one remainder item, and order them longest first, so a
// batch of consecutive items has similar sizes. Cached on the phantom per S.
koma_status ensure_items(koma_ctx* ctx, koma_phantom* ph, int S) {
    if (ph->items_s == S && ph->d_items) return KOMA_OK;
    const int64_t cap = 32LL * S;
    std::vector<int64_t> begin;
    std::vector<int32_t> gi(static_cast<size_t>(ph->n_groups + 1), 0);
    for (int64_t g = 0; g < ph->n_groups; ++g) {
        gi[g] = static_cast<int32_t>(begin.size());
        const int64_t lo = ph->group_offsets[g], n_g = ph->group_offsets[g + 1] - lo;
        for (int64_t off = 0; off < n_g; off += cap) begin.push_back(lo + off);
        if (begin.size() > static_cast<size_t>(std::numeric_limits<int32_t>::max() - 1))
            return fail(ctx, KOMA_E_INVALID, "simulate: grouped phantom needs too many work items");
    }
    gi[ph->n_groups] = static_cast<int32_t>(begin.size());
    const int64_t n_items = static_cast<int64_t>(begin.size());
    begin.push_back(ph->n);
    std::vector<int32_t> order(static_cast<size_t>(n_items));
    for (int64_t i = 0; i < n_items; ++i) order[i] = static_cast<int32_t>(i);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return begin[a + 1] - begin[a] > begin[b + 1] - begin[b];
    });
    if (ph->d_items) dev_free(ctx, ph->d_items, ph->items_bytes);
    ph->d_items = nullptr;
    ph->items_s = 0;
    const size_t b_items = begin.size() * sizeof(int64_t), b_order = order.size() * sizeof(int32_t),
                 b_gi = gi.size() * sizeof(int32_t);
    koma_status st = dev_alloc(ctx, reinterpret_cast<void**>(&ph->d_items), b_items + b_order + b_gi,
                               "simulate: work-item table");
    if (st != KOMA_OK) return st;
    ph->items_bytes = b_items + b_order + b_gi;
    ph->d_order = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ph->d_items) + b_items);
    ph->d_group_item = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ph->d_items) + b_items + b_order);
    cudaError_t e = h2d_sync(ctx, ph->d_items, begin.data(), b_items);
    if (e == cudaSuccess) e = h2d_sync(ctx, ph->d_order, order.data(), b_order);
    if (e == cudaSuccess) e = h2d_sync(ctx, ph->d_group_item, gi.data(), b_gi);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "simulate: work-item table copy");
    ph->n_items = n_items;
    ph->items_s = S;
    return KOMA_OK;
}

// K3z's work table: every group cut into units of up to 8 consecutive spins,
// units in group order, a warp taking 32 consecutive units; an item (one
// partial row) is the run of a warp's units that belong to one group, so a
// group's items are consecutive and K2 sums them in item order. Cached on the
// phantom (items_s = 8).
koma_status ensure_zunits(koma_ctx* ctx, koma_phantom* ph) {
    if (ph->items_s == 8 && ph->d_items) return KOMA_OK;
    constexpr int64_t kUnit = 8, kWarpUnits = 32;
    const int64_t G = ph->n_groups;
    // first unit and first item of every group: a group of m units has one
    // item plus one per warp start (a multiple of 32) strictly inside its units
    std::vector<int64_t> u0(static_cast<size_t>(G + 1), 0), i0(static_cast<size_t>(G + 1), 0);
    for (int64_t g = 0; g < G; ++g) {
        const int64_t m = (ph->group_offsets[g + 1] - ph->group_offsets[g] + kUnit - 1) / kUnit;
        u0[g + 1] = u0[g] + m;
        i0[g + 1] = i0[g] + (m > 0 ? 1 + (u0[g] + m - 1) / kWarpUnits - u0[g] / kWarpUnits : 0);
    }
    const int64_t n_units = u0[G], n_items = i0[G];
    if (n_items + 1 > std::numeric_limits<int32_t>::max())
        return fail(ctx, KOMA_E_INVALID, "simulate: grouped phantom needs too many work items");
    if (ph->d_items) dev_free(ctx, ph->d_items, ph->items_bytes);
    ph->d_items = nullptr;
    ph->items_s = 0;
    auto up16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t b_ub = static_cast<size_t>(n_units + 1) * sizeof(int64_t),
                 b_ui = up16(static_cast<size_t>(n_units) * sizeof(int32_t)),
                 b_gi = static_cast<size_t>(G + 1) * sizeof(int32_t);
    koma_status st = dev_alloc(ctx, reinterpret_cast<void**>(&ph->d_items), b_ub + b_ui + b_gi,
                               "simulate: unit table");
    if (st == KOMA_OK) st = stage_reserve(ctx, b_ub + b_ui + b_gi, 0);
    if (st != KOMA_OK) return st;
    ph->items_bytes = b_ub + b_ui + b_gi;
    ph->d_order = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ph->d_items) + b_ub);
    ph->d_group_item = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ph->d_items) + b_ub + b_ui);
    // the table, assembled in the pinned staging buffer (groups in parallel slices)
    int64_t* ub = reinterpret_cast<int64_t*>(ctx->h_stage);
    int32_t* ui = reinterpret_cast<int32_t*>(ctx->h_stage + b_ub);
    int32_t* gi = reinterpret_cast<int32_t*>(ctx->h_stage + b_ub + b_ui);
    const int k = n_units >= (int64_t{1} << 16) ? n_workers_for(16) : 1;
    run_tasks(k, [&](int w) {
        for (int64_t g = G * w / k; g < G * (w + 1) / k; ++g) {
            const int64_t lo = ph->group_offsets[g];
            gi[g] = static_cast<int32_t>(i0[g]);
            for (int64_t u = u0[g]; u < u0[g + 1]; ++u) {
                ub[u] = lo + (u - u0[g]) * kUnit;
                ui[u] = static_cast<int32_t>(i0[g] + u / kWarpUnits - u0[g] / kWarpUnits);
            }
        }
    });
    gi[G] = static_cast<int32_t>(n_items);
    ub[n_units] = ph->n;
    cudaError_t e = h2d_sync(ctx, ph->d_items, ctx->h_stage, b_ub + b_ui + b_gi);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "simulate: unit table copy");
    ph->n_items = n_items;
    ph->n_units = n_units;
    ph->items_s = 8;
    return KOMA_OK;
}

// The grouped kernel suits many small groups (dictionaries); a few large
// groups run faster through the CTA-split path.
bool use_items_kernel(const koma_phantom* ph) {
    return ph->n_groups > 1 && ph->n <= 512 * ph->n_groups;
}

// K3z's condition: spins that differ only in z (no x, y or off-resonance
// anywhere), a single T1 and T2 per group, and a stream without z gradients
// under RF or multi-sample ADC records.
bool z_dict_ok(const koma_phantom* ph, const koma_sequence* seq) {
    return ph->uni_relax && !ph->moving() && ph->max_abs[0] == 0 && ph->max_abs[1] == 0 && ph->max_abs[3] == 0 &&
           seq->z_dict && seq->r32z;
}

// K3z takes the phase as one FP32 product when |z Kz| <= 1 turn for every
// spin and record (its launches then use 128-thread CTAs).
bool z_small_phase(const koma_phantom* ph, const koma_sequence* seq) {
    return ph->max_abs[2] * seq->z_kmax <= 1.0;
}

koma_status grow_scratch(koma_ctx* ctx, size_t need, cudaStream_t st) {
    if (need <= ctx->scratch_bytes) return KOMA_OK;
    // the stream may still use the old buffer
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "simulate: sync before scratch growth");
    if (ctx->scratch) dev_free(ctx, ctx->scratch, ctx->scratch_bytes);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    koma_status s = dev_alloc(ctx, &ctx->scratch, need, "simulate: partial-sum scratch");
    if (s != KOMA_OK) return s;
    ctx->scratch_bytes = need;
    return KOMA_OK;
}

// Grouped kernel (K3) + per-group reduction (K2).
koma_status simulate_items(koma_ctx* ctx, koma_phantom* ph, const koma_sequence* seq, double* sig_dev,
                           cudaStream_t st, int S, int block, int tile) {
    // S == 8: K3z (items of 128 spins as for S = 4, two per warp)
    const bool zk = S == 8;
    if (zk && !z_dict_ok(ph, seq)) return fail(ctx, KOMA_E_INTERNAL, "simulate: K3z on an ineligible pair");
    koma_status rc = zk ? ensure_zunits(ctx, ph) : ensure_items(ctx, ph, S);
    if (rc != KOMA_OK) return rc;
    const int64_t n_adc = seq->info.n_adc;
    const bool small_phase = zk && z_small_phase(ph, seq);
    if (small_phase) block = std::min(block, 128);
    const int per_sm = std::max(1, zk ? koma::items_z_ctas_per_sm(block, tile, small_phase)
                                      : koma::items_ctas_per_sm(S, block, tile));
    // a batch is one item per warp (K3), or 32 units per warp (K3z)
    const int64_t per_batch = zk ? block : block / 32, work = zk ? ph->n_units : ph->n_items;
    const int64_t batches = (work + per_batch - 1) / per_batch;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(batches,
                                                         static_cast<int64_t>(ctx->sm_count) * per_sm)));
    rc = grow_scratch(ctx, static_cast<size_t>(ph->n_items) * static_cast<size_t>(n_adc) * 2 * sizeof(float), st);
    if (rc != KOMA_OK) return rc;
    koma::ItemArgs A;
    A.p32 = ph->p32;
    A.p64 = ph->p64;
    A.n_pad = ph->n_pad;
    A.item_begin = ph->d_items;
    A.order = ph->d_order;
    A.n_items = ph->n_items;
    A.counter = ctx->d_status + 1;
    A.rec = zk ? seq->r32z : seq->r32;
    A.n_rec = seq->info.n_records;
    A.partial = ctx->scratch;
    A.n_adc = n_adc;
    A.status = ctx->d_status;
    phantom_ext(ph, A.ext, &A.used);
    A.uni_relax = ph->uni_relax ? 1 : 0;
    if (zk) {
        A.unit_begin = ph->d_items;
        A.unit_item = ph->d_order;
        A.n_units = ph->n_units;
        A.item_begin = nullptr;
        A.order = nullptr;
    }
    cudaError_t ce = cudaMemsetAsync(A.counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "simulate: counter reset");
    if (ctx->timing) cudaEventRecord(ctx->ev[0], st);
    int e = zk ? koma::launch_items_z(A, grid, block, tile, small_phase, st)
               : koma::launch_items(A, grid, block, S, tile, st);
    if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate: grouped kernel launch");
    if (ctx->timing) {
        cudaEventRecord(ctx->ev[1], st);
        cudaEventRecord(ctx->ev[2], st);
    }
    koma::ReduceArgs R;
    R.partial = ctx->scratch;
    R.grid = static_cast<int>(ph->n_items);
    R.group_cta = ph->d_group_item;
    R.n_groups = ph->n_groups;
    R.n_adc = n_adc;
    R.sig = sig_dev;
    e = koma::launch_reduce(R, false, st);
    if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate: reduction launch");
    if (ctx->timing) {
        cudaEventRecord(ctx->ev[3], st);
        ctx->timing_recorded = true;
    }
    ctx->last.kernels = 2;
    ctx->last.grid = grid;
    ctx->last.block = block;
    ctx->last.spins_per_thread = S;
    ctx->last.spins_per_cta = 32LL * S * (block / 32);
    ctx->last.n_records = seq->info.n_records;
    ctx->last.partial_bytes = static_cast<int64_t>(ph->n_items * n_adc * 8);
    ctx->last.split = 1;
    ctx->last.tile_records = tile;
    ctx->last.phase_mode = small_phase ? 1 : 0;
    return KOMA_OK;
}

// Shape bucket of a launch for the autotuner cache: the kernel family
// (grouped items, K3z with either phase, FP32 Bloch, motion), and the powers
// of two of the spins, groups, records and ADC samples.
uint64_t tune_key(const koma_phantom* ph, const koma_sequence* seq, bool items) {
    auto lg = [](int64_t v) { return static_cast<uint64_t>(v > 0 ? 64 - __builtin_clzll(static_cast<uint64_t>(v)) : 0); };
    const bool z = items && z_dict_ok(ph, seq);
    const uint64_t family = items ? (z ? (z_small_phase(ph, seq) ? 4 : 3) : 1) : (ph->moving() ? 2 : 0);
    return family | lg(ph->n) << 3 | lg(ph->n_groups) << 11 | lg(seq->info.n_records) << 19 |
           lg(seq->info.n_adc) << 27 | lg(seq->info.n_rf) << 35;
}

// Largest snapshot buffer (8 bytes per spin and block of matrix-form runs)
// the tensor-core readout takes; beyond it the Bloch kernel samples every
// run itself.
constexpr size_t kMmaMaxEBytes = size_t{16} << 30;
// Largest buffer of repeated-pulse maps (48 bytes per spin and pulse).
constexpr size_t kRfMapMaxBytes = size_t{16} << 30;

// ADC-run split for a launch whose spins fill few warps: CTAs sharing a
// spin range each take every split-th ADC record (all of them step the RF
// and PREC records), up to about 16 resident warps per SM. Only when
// sampling dominates the work (the RF steps are repeated by every part) and
// there are enough runs to share.
int choose_split(const koma_ctx* ctx, const koma::BlochLaunch& L, const koma_sequence* seq) {
    const int64_t warps = static_cast<int64_t>(L.grid) * ((L.block + 31) / 32);
    const int64_t target = static_cast<int64_t>(ctx->sm_count) * 16;
    if (50 * seq->info.n_rf > 8 * seq->info.n_adc) return 1;
    int split = 1;
    while (split < 8 && warps * split * 2 <= target && seq->info.n_adc_runs >= 8 * split) split *= 2;
    return split;
}

// Launch shape: the grid is a whole number of waves of (SMs x resident CTAs)
// and every CTA gets the same number of spins, so no SM idles on a tail.
koma::BlochLaunch choose_launch(const koma_ctx* ctx, int64_t n, bool fp64, int s_fp32 = 4, bool moving = false) {
    koma::BlochLaunch L;
    const int S = fp64 ? 1 : (moving ? koma::kMotionSpinsPerThread : s_fp32);
    const int max_block = koma::bloch_max_block();
    const int per_sm = std::max(1, moving && !fp64 ? koma::motion_ctas_per_sm(max_block)
                                                   : koma::bloch_ctas_per_sm(fp64, S, max_block));
    const int64_t slots = static_cast<int64_t>(ctx->sm_count) * per_sm;
    const int64_t wave_spins = slots * max_block * S;
    const int64_t waves = std::max<int64_t>(1, (n + wave_spins - 1) / wave_spins);
    int64_t grid = slots * waves;
    int64_t spc = std::max<int64_t>(1, (n + grid - 1) / grid);
    grid = std::max<int64_t>(1, (n + spc - 1) / spc);
    const int64_t threads = (spc + S - 1) / S;
    L.block = static_cast<int>(std::min<int64_t>(max_block, std::max<int64_t>(32, (threads + 31) / 32 * 32)));
    L.grid = static_cast<int>(grid);
    L.spins_per_thread = S;
    L.spins_per_cta = spc;
    return L;
}

}  // namespace

extern "C" koma_status koma_simulate(koma_ctx* ctx, const koma_phantom* ph_c, const koma_sequence* seq,
                                     koma_precision precision, double* sig_dev, void* stream) {
    NvtxRange nvtx_("koma_simulate");
    if (!ctx) return KOMA_E_INVALID;
    koma_phantom* ph = const_cast<koma_phantom*>(ph_c);
    if (!ph || !seq) return fail(ctx, KOMA_E_INVALID, "simulate: NULL phantom or sequence");
    if (ph->ctx != ctx || seq->ctx != ctx)
        return fail(ctx, KOMA_E_INVALID, "simulate: phantom/sequence belong to another context");
    if (precision != KOMA_FP64 && precision != KOMA_FP32_SPLITPHASE)
        return fail(ctx, KOMA_E_INVALID, "simulate: unknown precision %d", static_cast<int>(precision));
    const int64_t n_adc = seq->info.n_adc;
    if (n_adc > 0 && !sig_dev) return fail(ctx, KOMA_E_INVALID, "simulate: sig_dev is NULL");
    const bool fp64 = precision == KOMA_FP64;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, KOMA_E_CUDA, "simulate: cannot select device %d", ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->last = koma_launch_info{};
    ctx->last.bloch_stream = stream;
    if (n_adc == 0) return KOMA_OK;  // nothing is observed
    const int64_t out_bytes = n_adc * ph->n_groups * 2 * static_cast<int64_t>(sizeof(double));
    if (ph->n == 0) {
        cudaError_t e = cudaMemsetAsync(sig_dev, 0, static_cast<size_t>(out_bytes), st);
        return e == cudaSuccess ? KOMA_OK : cuda_fail(ctx, e, "simulate: memset");
    }

    const bool moving = ph->moving();
    if (!fp64 && !moving && use_items_kernel(ph)) {
        const bool tuned = ph->tuned_seq == seq && ph->tuned_n_rec == seq->info.n_records;
        // untuned default: the tuner's usual pick for dictionaries of small
        // groups, K3z where it applies
        const bool zk = z_dict_ok(ph, seq);
        int S = tuned ? ph->tuned_s : (zk ? 8 : 2), block = tuned ? ph->tuned_block : 128;
        int tile = tuned && ph->tuned_tile > 0 ? ph->tuned_tile : (zk ? 128 : 64);
        if (!tuned) {
            auto it = ctx->tune_cache.find(tune_key(ph, seq, true));
            if (it != ctx->tune_cache.end()) {
                S = it->second.s;
                block = it->second.block;
                tile = it->second.tile;
            }
        }
        ctx->timing_recorded = false;
        ctx->maps_timed = false;
        return simulate_items(ctx, ph, seq, sig_dev, st, S, block, tile);
    }
    const bool tuned_k1 = ph->tuned_seq == seq && ph->tuned_n_rec == seq->info.n_records && ph->tuned_s > 0;
    int s_k1 = tuned_k1 ? ph->tuned_s : 4;
    if (!tuned_k1 && !fp64) {
        auto it = ctx->tune_cache.find(tune_key(ph, seq, false));
        if (it != ctx->tune_cache.end()) s_k1 = it->second.s;
    }
    koma::BlochLaunch L = choose_launch(ctx, ph->n, fp64, s_k1, moving);
    if (ph->n_groups > 1) {
        // size CTAs for the largest group (groups never share a CTA)
        int64_t gmax = 1;
        for (int64_t gi = 0; gi < ph->n_groups; ++gi)
            gmax = std::max(gmax, ph->group_offsets[gi + 1] - ph->group_offsets[gi]);
        if (gmax < L.spins_per_cta) {
            L.spins_per_cta = gmax;
            const int64_t threads = (gmax + L.spins_per_thread - 1) / L.spins_per_thread;
            L.block = static_cast<int>(std::max<int64_t>(32, (threads + 31) / 32 * 32));
        }
    }
    if (fp64) {
        L.spins_per_thread = 1;
        L.block = static_cast<int>(std::min<int64_t>(L.block, koma::bloch_max_block()));
        L.spins_per_cta = std::min<int64_t>(L.spins_per_cta, L.block);
        L.grid = static_cast<int>((ph->n + L.spins_per_cta - 1) / L.spins_per_cta);
    }
    const int split = (!fp64 && ph->n_groups == 1) ? choose_split(ctx, L, seq) : 1;
    L.grid *= split;
    koma::BlochArgs A;
    A.split = split;
    A.p32 = ph->p32;
    A.p64 = ph->p64;
    A.n_pad = ph->n_pad;
    A.n = ph->n;
    if ((fp64 && !seq->r64) || (moving && !fp64 && !seq->rm))
        return fail(ctx, KOMA_E_INVALID, "simulate: the sequence was uploaded without its %s records",
                    fp64 ? "FP64" : "motion");
    A.rec = fp64 ? static_cast<const void*>(seq->r64)
                 : (moving ? static_cast<const void*>(seq->rm) : static_cast<const void*>(seq->r32));
    A.n_rec = seq->info.n_records;
    A.n_adc = n_adc;
    A.status = ctx->d_status;
    phantom_ext(ph, A.ext, &A.used);
    if (moving) motion_args(ph, A);
    A.spins_per_cta = L.spins_per_cta;
    koma::ReduceArgs R;
    R.n_adc = n_adc;
    R.n_groups = ph->n_groups;

    if (ph->n_groups > 1) {
        // CTAs never straddle a group: each group gets ceil(n_g / spc) CTAs
        if (ph->cfg_spc != L.spins_per_cta) {
            // h[c] = first spin of CTA c; CTA c owns [h[c], h[c+1]). The last
            // CTA of a group ends where the next non-empty group begins, so
            // the begins alone describe the split (h[grid] = n).
            std::vector<int64_t> h;
            std::vector<int32_t> gc(static_cast<size_t>(ph->n_groups + 1), 0);
            for (int64_t gi = 0; gi < ph->n_groups; ++gi) {
                gc[gi] = static_cast<int32_t>(h.size());
                for (int64_t s0 = ph->group_offsets[gi]; s0 < ph->group_offsets[gi + 1]; s0 += L.spins_per_cta)
                    h.push_back(s0);
                if (h.size() > static_cast<size_t>(std::numeric_limits<int32_t>::max() - 1))
                    return fail(ctx, KOMA_E_INVALID, "simulate: grouped launch needs too many CTAs");
            }
            gc[ph->n_groups] = static_cast<int32_t>(h.size());
            const size_t n_cta = h.size();
            h.push_back(ph->n);
            if (ph->d_cta_begin) dev_free(ctx, ph->d_cta_begin, ph->table_bytes);
            ph->d_cta_begin = nullptr;
            ph->d_group_cta = nullptr;
            const size_t tbytes = h.size() * sizeof(int64_t) + gc.size() * sizeof(int32_t);
            koma_status s = dev_alloc(ctx, reinterpret_cast<void**>(&ph->d_cta_begin), tbytes, "simulate: CTA table");
            if (s != KOMA_OK) return s;
            ph->table_bytes = tbytes;
            ph->d_group_cta = reinterpret_cast<int32_t*>(ph->d_cta_begin + h.size());
            cudaError_t e = h2d_sync(ctx, ph->d_cta_begin, h.data(), h.size() * sizeof(int64_t));
            if (e == cudaSuccess) e = h2d_sync(ctx, ph->d_group_cta, gc.data(), gc.size() * sizeof(int32_t));
            if (e != cudaSuccess) return cuda_fail(ctx, e, "simulate: CTA table copy");
            ph->grid = static_cast<int>(n_cta);
            ph->cfg_spc = L.spins_per_cta;
        }
        L.grid = ph->grid;
        A.cta_begin = ph->d_cta_begin;
        R.group_cta = ph->d_group_cta;
    }

    const size_t elem = fp64 ? 2 * sizeof(double) : 2 * sizeof(float);
    const int rows = L.grid / split;  // one partial row per spin range
    size_t need = static_cast<size_t>(rows) * static_cast<size_t>(n_adc) * elem;
    // tensor-core readout of the sequence's matrix-form groups: scratch
    // [Bloch rows | readout rows (grid_mma x n_adc float2) | snapshots (n_mma_snaps x n_pad float2)]
    const size_t e_bytes = static_cast<size_t>(seq->n_mma_snaps) * static_cast<size_t>(ph->n_pad) * sizeof(float2);
    const bool use_mma = !fp64 && !moving && ph->n_groups == 1 && seq->n_mma_groups > 0 && ctx->mma_enabled &&
                         e_bytes <= kMmaMaxEBytes;
    int grid_mma = 0;
    int64_t spc_mma = 0;
    size_t off_rows = 0, off_e = 0;
    if (use_mma) {
        // every CTA gets at least one block of 32 spins (each writes its whole row)
        const int64_t blocks = (ph->n + 31) / 32;
        int64_t g6 = std::min<int64_t>(ctx->sm_count, blocks);
        const int64_t per_cta = (blocks + g6 - 1) / g6;
        g6 = (blocks + per_cta - 1) / per_cta;
        grid_mma = static_cast<int>(g6);
        spc_mma = per_cta * 32;
        auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
        off_rows = up256(need);
        off_e = up256(off_rows + static_cast<size_t>(grid_mma) * static_cast<size_t>(n_adc) * sizeof(float2));
        need = off_e + e_bytes;
    }
    // maps of repeated RF pulses (FP32 static Bloch kernel): scratch
    // [n_maps][3][n_pad] float4 after the rest, at most kRfMapMaxBytes
    const size_t map_bytes = static_cast<size_t>(koma::kRfMapFloats) * static_cast<size_t>(ph->n_pad) * sizeof(float);
    int n_maps = 0;
    size_t off_maps = 0;
    // all of the sequence's maps or none (the compacted stream stands for all)
    if (!fp64 && !moving && ctx->rf_maps_enabled && seq->n_rf_maps > 0 &&
        static_cast<size_t>(seq->n_rf_maps) * map_bytes <= kRfMapMaxBytes) {
        n_maps = seq->n_rf_maps;
        off_maps = (need + 255) / 256 * 256;
        need = off_maps + static_cast<size_t>(n_maps) * map_bytes;
    }
    {
        koma_status s = grow_scratch(ctx, need, st);
        if (s != KOMA_OK) return s;
    }
    A.partial = ctx->scratch;
    koma::RfMapArgs F;
    if (n_maps > 0) {
        F.p32 = ph->p32;
        F.n_pad = ph->n_pad;
        F.n = ph->n;
        F.rec = seq->r32;
        F.pulses = seq->d_rf_pulses;
        F.n_pulses = n_maps;
        F.maps = reinterpret_cast<float*>(static_cast<char*>(ctx->scratch) + off_maps);
        for (int d = 0; d < 4; ++d) F.ext[d] = A.ext[d];
        A.rf_maps = F.maps;
        A.n_rf_maps = n_maps;
        A.rec = seq->r32c;
        A.n_rec = seq->n_rec_c;
    }
    R.partial = ctx->scratch;
    R.grid = rows;
    R.sig = sig_dev;
    koma::MmaArgs M;
    if (use_mma) {
        char* base = static_cast<char*>(ctx->scratch);
        A.mma_snap = reinterpret_cast<float2*>(base + off_e);
        A.n_mma_snaps = seq->n_mma_snaps;
        M.p32 = ph->p32;
        M.n_pad = ph->n_pad;
        M.n = ph->n;
        M.snap = A.mma_snap;
        M.used = A.used;
        M.groups = seq->d_mma_groups;
        M.n_groups = seq->n_mma_groups;
        M.runs = seq->d_mma_runs;
        M.partial = reinterpret_cast<float2*>(base + off_rows);
        M.n_adc = n_adc;
        M.spins_per_cta = spc_mma;
        // |Mxy| <= about max pd: scale E by a power of two below 1/max pd
        // (exact) so its FP16 parts stay in range; undone on the result
        int ex = 0;
        if (ph->max_pd > 0) std::frexp(ph->max_pd, &ex);
        ex = std::max(-100, std::min(100, ex));
        A.mma_escale = std::ldexp(1.0f, -ex);
        M.einv = std::ldexp(1.0f, ex);
        M.status = ctx->d_status;
        R.partial_mma = M.partial;
        R.grid_mma = grid_mma;
        R.from_mma = seq->d_from_mma;
    }

    ctx->timing_recorded = false;

    ctx->maps_timed = false;
    if (ctx->timing) cudaEventRecord(ctx->ev[0], st);
    int e;
    if (n_maps > 0) {
        e = koma::launch_rf_maps(F, stream);
        if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate: pulse-map launch");
        if (ctx->timing) {
            cudaEventRecord(ctx->ev_maps, st);
            ctx->maps_timed = true;
        }
    }
    if (moving)
        e = fp64 ? koma::launch_bloch_fp64_motion(A, L, stream) : koma::launch_bloch_motion(A, L, stream);
    else
        e = fp64 ? koma::launch_bloch_fp64(A, L, stream) : koma::launch_bloch_fp32(A, L, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate: Bloch kernel launch");
    if (ctx->timing) cudaEventRecord(ctx->ev[1], st);
    if (use_mma) {
        e = koma::launch_readout_mma(M, grid_mma, stream);
        if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate: readout launch");
    }
    if (ctx->timing) cudaEventRecord(ctx->ev[2], st);
    e = koma::launch_reduce(R, fp64, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate: reduction launch");
    if (ctx->timing) {
        cudaEventRecord(ctx->ev[3], st);
        ctx->timing_recorded = true;
    }

    ctx->last.kernels = (use_mma ? 3 : 2) + (n_maps > 0 ? 1 : 0);
    ctx->last.mma_grid = grid_mma;
    ctx->last.grid = L.grid;
    ctx->last.block = L.block;
    ctx->last.spins_per_thread = L.spins_per_thread;
    ctx->last.spins_per_cta = L.spins_per_cta;
    ctx->last.n_records = A.n_rec;
    ctx->last.partial_bytes = static_cast<int64_t>(need);
    ctx->last.split = split;
    ctx->last.tile_records = moving ? 64 : (fp64 ? 0 : 256);
    return KOMA_OK;
}

// Allocation-free variant of koma_simulate (FP32 split-phase path): the
// per-CTA partial sums go to the library's static device array instead of
// the context's cudaMalloc'ed scratch. Ungrouped phantoms only (a grouped
// launch needs a device CTA table). Allocates nothing.
extern "C" koma_status koma_simulate_static(const koma_phantom* ph, const koma_sequence* seq, double* sig_dev,
                                            void* stream) {
    NvtxRange nvtx_("koma_simulate_static");
    if (!ph || !seq) return KOMA_E_INVALID;
    koma_ctx* ctx = ph->ctx;
    if (seq->ctx != ctx) return fail(ctx, KOMA_E_INVALID, "simulate_static: phantom and sequence belong to different contexts");
    if (ph->n_groups > 1)
        return fail(ctx, KOMA_E_INVALID, "simulate_static: grouped phantoms are not supported (use koma_simulate)");
    if (ph->moving())
        return fail(ctx, KOMA_E_INVALID, "simulate_static: moving phantoms are not supported (use koma_simulate)");
    const int64_t n_adc = seq->info.n_adc;
    if (n_adc == 0) return KOMA_OK;
    if (!sig_dev) return fail(ctx, KOMA_E_INVALID, "simulate_static: sig_dev is NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, KOMA_E_CUDA, "simulate_static: cannot select device %d", ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the launch description and stage timing describe this call from here on
    // (the static path records no stage events)
    ctx->last = koma_launch_info{};
    ctx->last.bloch_stream = stream;
    ctx->timing_recorded = false;
    ctx->maps_timed = false;
    if (ph->n == 0) {
        cudaError_t e = cudaMemsetAsync(sig_dev, 0, static_cast<size_t>(n_adc) * 2 * sizeof(double), st);
        return e == cudaSuccess ? KOMA_OK : cuda_fail(ctx, e, "simulate_static: memset");
    }
    void* scratch = nullptr;
    int ce = koma::static_partials_ptr(ctx->device, &scratch);
    if (ce != cudaSuccess)
        return cuda_fail(ctx, static_cast<cudaError_t>(ce), "simulate_static: static scratch address");
    const int64_t cap = static_cast<int64_t>(koma::static_partials_capacity());
    koma::BlochLaunch L = choose_launch(ctx, ph->n, false);
    if (static_cast<int64_t>(L.grid) * n_adc > cap) {
        // fewest CTAs: every thread full
        const int64_t spc = static_cast<int64_t>(koma::bloch_max_block()) * L.spins_per_thread;
        L.spins_per_cta = spc;
        L.grid = static_cast<int>((ph->n + spc - 1) / spc);
        L.block = koma::bloch_max_block();
    }
    if (static_cast<int64_t>(L.grid) * n_adc > cap)
        return fail(ctx, KOMA_E_INVALID,
                    "simulate_static: %lld spins x %lld ADC samples need %lld partial sums; the static scratch "
                    "holds %lld (use koma_simulate)",
                    static_cast<long long>(ph->n), static_cast<long long>(n_adc),
                    static_cast<long long>(L.grid) * n_adc, static_cast<long long>(cap));
    koma::BlochArgs A;
    A.p32 = ph->p32;
    A.p64 = ph->p64;
    A.n_pad = ph->n_pad;
    A.n = ph->n;
    A.rec = seq->r32;
    A.n_rec = seq->info.n_records;
    A.n_adc = n_adc;
    A.status = ctx->d_status;
    phantom_ext(ph, A.ext, &A.used);
    A.spins_per_cta = L.spins_per_cta;
    A.partial = scratch;  // every (CTA, sample) entry is written before K2 reads it
    koma::ReduceArgs R;
    R.n_adc = n_adc;
    R.n_groups = 1;
    R.partial = scratch;
    R.grid = L.grid;
    R.sig = sig_dev;
    int e = koma::launch_bloch_fp32(A, L, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate_static: Bloch kernel launch");
    e = koma::launch_reduce(R, false, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, static_cast<cudaError_t>(e), "simulate_static: reduction launch");
    ctx->last.kernels = 2;
    ctx->last.grid = L.grid;
    ctx->last.block = L.block;
    ctx->last.spins_per_thread = L.spins_per_thread;
    ctx->last.spins_per_cta = L.spins_per_cta;
    ctx->last.n_records = seq->info.n_records;
    ctx->last.partial_bytes = static_cast<int64_t>(L.grid) * n_adc * static_cast<int64_t>(sizeof(float2));
    ctx->last.split = 1;
    ctx->last.tile_records = 256;
    return KOMA_OK;
}

extern "C" koma_status koma_tune(koma_ctx* ctx, const koma_phantom* ph_c, const koma_sequence* seq,
                                 double* sig_dev, void* stream, koma_launch_info* chosen) {
    NvtxRange nvtx_("koma_tune");
    if (!ctx) return KOMA_E_INVALID;
    koma_phantom* ph = const_cast<koma_phantom*>(ph_c);
    if (!ph || !seq) return fail(ctx, KOMA_E_INVALID, "tune: NULL phantom or sequence");
    if (ph->ctx != ctx || seq->ctx != ctx) return fail(ctx, KOMA_E_INVALID, "tune: objects of another context");
    if (seq->info.n_adc > 0 && !sig_dev) return fail(ctx, KOMA_E_INVALID, "tune: sig_dev is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    struct Cand {
        int s, block, tile;
    };
    std::vector<Cand> cands;
    const bool items = !ph->moving() && use_items_kernel(ph);
    if (ph->moving()) {
        cands = {{koma::kMotionSpinsPerThread, 0, 0}};  // one motion kernel shape
    } else if (items) {
        // spins per thread x CTA size x sequence-tile length
        for (int s_ : {2, 4})
            for (int b_ : {128, 256})
                for (int t_ : {64, 128, 256}) cands.push_back({s_, b_, t_});
        if (z_dict_ok(ph, seq))
            for (int b_ : {128, 256})
                for (int t_ : {128, 256})
                    if (b_ == 128 || !z_small_phase(ph, seq)) cands.push_back({8, b_, t_});
    } else {
        cands = {{2, 0, 0}, {4, 0, 0}};
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(ctx, KOMA_E_CUDA, "tune: event creation");
    float best = -1.f;
    Cand pick = cands.back();
    koma_status rc = KOMA_OK;
    for (size_t i = 0; i < cands.size() && rc == KOMA_OK; ++i) {
        ph->tuned_seq = seq;
        ph->tuned_n_rec = seq->info.n_records;
        ph->tuned_s = cands[i].s;
        ph->tuned_block = cands[i].block;
        ph->tuned_tile = cands[i].tile;
        // one untimed run (tables, scratch), one timed
        for (int rep = 0; rep < 2 && rc == KOMA_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, st);
            rc = koma_simulate(ctx, ph, seq, KOMA_FP32_SPLITPHASE, sig_dev, stream);
            if (rep == 1) cudaEventRecord(e1, st);
        }
        if (rc != KOMA_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(ctx, KOMA_E_CUDA, "tune: event wait");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0.f || ms < best) {
            best = ms;
            pick = cands[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != KOMA_OK) {
        ph->tuned_seq = nullptr;
        return rc;
    }
    ph->tuned_seq = seq;
    ph->tuned_n_rec = seq->info.n_records;
    ph->tuned_s = pick.s;
    ph->tuned_block = pick.block;
    ph->tuned_tile = pick.tile;
    ctx->tune_cache[tune_key(ph, seq, items)] = {pick.s, pick.block, pick.tile};
    if (chosen) {
        rc = koma_simulate(ctx, ph, seq, KOMA_FP32_SPLITPHASE, sig_dev, stream);
        *chosen = ctx->last;
    }
    return rc;
}

extern "C" koma_status koma_check_bounded_wait(koma_ctx* ctx, int64_t limit_us, void* stream) {
    if (!ctx) return KOMA_E_INVALID;
    if (limit_us < 1 || limit_us > 2000000)
        return fail(ctx, KOMA_E_INVALID, "check_bounded_wait: limit_us = %lld (1 .. 2,000,000)",
                    static_cast<long long>(limit_us));
    DeviceGuard g(ctx->device);
    int e = koma::launch_bounded_wait_check(ctx->d_status, static_cast<unsigned long long>(limit_us) * 1000ull,
                                            stream);
    return e == cudaSuccess ? KOMA_OK : cuda_fail(ctx, static_cast<cudaError_t>(e), "check_bounded_wait: launch");
}

extern "C" koma_status koma_sync(koma_ctx* ctx, void* stream) {
    if (!ctx) return KOMA_E_INVALID;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync");
    int flag = 0;
    // the status word, read and cleared on the context's stream (ordered
    // with everything the caller's stream ran before: it was synchronised)
    e = cudaMemcpyAsync(&flag, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->own_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->own_stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sync: status read");
    if (flag) {
        memset_sync(ctx, ctx->d_status, 0, sizeof(int));
        if (flag & (koma::kStatusTimeout | koma::kStatusWaitCheck))
            return fail(ctx, KOMA_E_TIMEOUT, "a bounded device-side wait gave up (status 0x%x)", flag);
        return fail(ctx, KOMA_E_INTERNAL,
                    "a kernel met a record outside its launch's buffers and skipped it (status 0x%x:%s%s%s%s)",
                    flag, (flag & koma::kStatusBadAdc) ? " ADC run" : "", (flag & koma::kStatusBadMap) ? " map slot" : "",
                    (flag & koma::kStatusBadSnap) ? " snapshot row" : "",
                    (flag & koma::kStatusBadRun) ? " readout run" : "");
    }
    return KOMA_OK;
}

extern "C" koma_status koma_set_timing(koma_ctx* ctx, int enable) {
    if (!ctx) return KOMA_E_INVALID;
    DeviceGuard g(ctx->device);
    if (enable && !ctx->ev[0]) {
        for (cudaEvent_t& e : ctx->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(ctx, r, "set_timing: event");
        }
        cudaError_t r = cudaEventCreate(&ctx->ev_maps);
        if (r != cudaSuccess) return cuda_fail(ctx, r, "set_timing: event");
    }
    ctx->timing = enable != 0;
    ctx->timing_recorded = false;
    ctx->maps_timed = false;
    return KOMA_OK;
}

extern "C" koma_status koma_get_timing(koma_ctx* ctx, float* bloch_ms, float* reduce_ms) {
    if (!ctx || !bloch_ms || !reduce_ms) return KOMA_E_INVALID;
    if (!ctx->timing_recorded) return fail(ctx, KOMA_E_INVALID, "get_timing: no timed simulate call");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(bloch_ms, ctx->ev[0], ctx->ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(reduce_ms, ctx->ev[2], ctx->ev[3]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_timing");
    return KOMA_OK;
}

extern "C" koma_status koma_get_stage_timing(koma_ctx* ctx, float* bloch_ms, float* mma_ms, float* reduce_ms) {
    if (!ctx || !bloch_ms || !mma_ms || !reduce_ms) return KOMA_E_INVALID;
    if (!ctx->timing_recorded) return fail(ctx, KOMA_E_INVALID, "get_stage_timing: no timed simulate call");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(bloch_ms, ctx->ev[0], ctx->ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(mma_ms, ctx->ev[1], ctx->ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(reduce_ms, ctx->ev[2], ctx->ev[3]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_stage_timing");
    return KOMA_OK;
}

extern "C" koma_status koma_set_mma(koma_ctx* ctx, int enable) {
    if (!ctx) return KOMA_E_INVALID;
    ctx->mma_enabled = enable != 0;
    return KOMA_OK;
}

extern "C" koma_status koma_set_rf_maps(koma_ctx* ctx, int enable) {
    if (!ctx) return KOMA_E_INVALID;
    ctx->rf_maps_enabled = enable != 0;
    return KOMA_OK;
}

extern "C" koma_status koma_get_map_timing(koma_ctx* ctx, float* maps_ms) {
    if (!ctx || !maps_ms) return KOMA_E_INVALID;
    if (!ctx->timing_recorded) return fail(ctx, KOMA_E_INVALID, "get_map_timing: no timed simulate call");
    *maps_ms = 0.f;
    if (!ctx->maps_timed) return KOMA_OK;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->ev[3]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(maps_ms, ctx->ev[0], ctx->ev_maps);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_map_timing");
    return KOMA_OK;
}

extern "C" koma_status koma_get_launch_info(const koma_ctx* ctx, koma_launch_info* info) {
    if (!ctx || !info) return KOMA_E_INVALID;
    *info = ctx->last;
    return KOMA_OK;
}

namespace {

// A host-buffer simulation in two halves, so that a batch can run one job's
// host work while the device simulates the previous one: start = checks,
// uploads (the phantom's copies and conversion on the device while the host
// preprocesses the sequence), the simulation and the signal's copy-back
// enqueued on the context's stream; finish = wait, then the stream-ordered
// frees.
struct HostJob {
    koma_phantom* ph = nullptr;
    koma_sequence* seq = nullptr;
    double* d_sig = nullptr;
    size_t out_bytes = 0;
    bool active = false;
};

koma_status host_job_finish(koma_ctx* ctx, HostJob& J, koma_status st) {
    if (!J.active) return st;
    DeviceGuard g(ctx->device);
    if (st == KOMA_OK) st = koma_sync(ctx, ctx->own_stream);
    // every use of these blocks was on own_stream: frees ordered there
    dev_free_on(ctx, J.d_sig, J.out_bytes, ctx->own_stream);
    koma::sequence_free_on(J.seq, ctx->own_stream);
    koma::phantom_free_on(J.ph, ctx->own_stream);
    J = HostJob{};
    return st;
}

// `after`: an event the simulation waits for (a batch runs its jobs' device
// work one after another: two simulations sharing the GPU slow each other
// down more than they gain); `done`: recorded after the simulation, before
// the signal's copy-back.
koma_status host_job_start(koma_ctx* ctx, const koma_host_job& j, koma_precision precision, HostJob& J,
                           cudaEvent_t after = nullptr, cudaEvent_t done = nullptr) {
    J = HostJob{};
    J.active = true;
    koma_status st = phantom_upload_start(ctx, j.n, j.x, j.y, j.z, j.pd, j.t1, j.t2, j.dw, j.group_offsets,
                                          j.n_groups, &J.ph);
    // the phantom is static here: no motion records; FP64 records only for the FP64 path
    if (st == KOMA_OK)
        st = sequence_upload_impl(ctx, j.n_steps, j.dt, j.gx, j.gy, j.gz, j.b1_re, j.b1_im, j.adc,
                                  precision == KOMA_FP64, false, &J.seq);
    if (J.ph) {
        const koma_status sp = phantom_upload_finish(ctx, &J.ph, j.x, j.y, j.z, j.pd, j.t1, j.t2, j.dw);
        if (st == KOMA_OK) st = sp;
    }
    DeviceGuard g(ctx->device);
    if (st == KOMA_OK) {
        J.out_bytes = static_cast<size_t>(J.seq->info.n_adc * J.ph->n_groups) * 2 * sizeof(double);
        if (J.out_bytes && !j.sig_host) st = fail(ctx, KOMA_E_INVALID, "simulate_host: sig_host is NULL");
    }
    if (st == KOMA_OK)
        st = dev_alloc(ctx, reinterpret_cast<void**>(&J.d_sig), J.out_bytes, "simulate_host: signal");
    if (st == KOMA_OK && after) {
        const cudaError_t e = cudaStreamWaitEvent(ctx->own_stream, after, 0);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "simulate_host: ordering after the previous job");
    }
    if (st == KOMA_OK) st = koma_simulate(ctx, J.ph, J.seq, precision, J.d_sig, ctx->own_stream);
    if (st == KOMA_OK && done) {  // before the copy-back, which overlaps the next job's simulation
        const cudaError_t e = cudaEventRecord(done, ctx->own_stream);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "simulate_host: job event");
    }
    if (st == KOMA_OK && J.out_bytes) {
        cudaError_t e = cudaMemcpyAsync(j.sig_host, J.d_sig, J.out_bytes, cudaMemcpyDeviceToHost, ctx->own_stream);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "simulate_host: copy back");
    }
    return st;
}

}  // namespace

extern "C" koma_status koma_simulate_host(koma_ctx* ctx, int64_t n, const double* x, const double* y,
                                          const double* z, const double* pd, const double* t1, const double* t2,
                                          const double* dw, const int64_t* group_offsets, int64_t n_groups,
                                          int64_t n_steps, const double* dt, const double* gx, const double* gy,
                                          const double* gz, const double* b1_re, const double* b1_im,
                                          const uint8_t* adc, koma_precision precision, double* sig_host) {
    NvtxRange nvtx_("koma_simulate_host");
    if (!ctx) return KOMA_E_INVALID;
    const koma_host_job j{n, x, y, z, pd, t1, t2, dw, group_offsets, n_groups, n_steps,
                          dt, gx, gy, gz, b1_re, b1_im, adc, sig_host};
    HostJob J;
    const koma_status st = host_job_start(ctx, j, precision, J);
    return host_job_finish(ctx, J, st);
}

extern "C" koma_status koma_simulate_host_batch(koma_ctx* ctx, int64_t n_jobs, const koma_host_job* jobs,
                                                koma_precision precision) {
    NvtxRange nvtx_("koma_simulate_host_batch");
    if (!ctx) return KOMA_E_INVALID;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, KOMA_E_INVALID, "simulate_host_batch: bad job list");
    if (n_jobs > 1 && !ctx->twin) {
        const koma_status ti = koma_init(ctx->device, ctx->budget, &ctx->twin);
        if (ti != KOMA_OK) {
            ctx->twin = nullptr;
            return fail(ctx, ti, "simulate_host_batch: second context: cannot create it");
        }
    }
    if (ctx->twin) {  // the second context simulates as ctx would: its switches and tuned shapes
        ctx->twin->mma_enabled = ctx->mma_enabled;
        ctx->twin->rf_maps_enabled = ctx->rf_maps_enabled;
        ctx->twin->tune_cache = ctx->tune_cache;
    }
    koma_ctx* c[2] = {ctx, ctx->twin ? ctx->twin : ctx};
    for (koma_ctx* x : c) {
        DeviceGuard g(x->device);
        if (!x->ev_job && cudaEventCreateWithFlags(&x->ev_job, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            x->ev_job = nullptr;
            return fail(ctx, KOMA_E_CUDA, "simulate_host_batch: event creation");
        }
    }
    HostJob J[2];
    koma_status st = KOMA_OK;
    int failed = 0;
    for (int64_t i = 0; i < n_jobs && st == KOMA_OK; ++i) {
        const int k = static_cast<int>(i & 1);
        st = host_job_finish(c[k], J[k], KOMA_OK);  // the job this context ran two jobs ago
        // this job's device work follows the previous job's
        if (st == KOMA_OK)
            st = host_job_start(c[k], jobs[i], precision, J[k], i > 0 ? c[k ^ 1]->ev_job : nullptr, c[k]->ev_job);
        if (st != KOMA_OK) failed = k;
    }
    for (int k = 0; k < 2; ++k) {
        const koma_status sk = host_job_finish(c[k], J[k], KOMA_OK);
        if (st == KOMA_OK && sk != KOMA_OK) {
            st = sk;
            failed = k;
        }
    }
    if (st != KOMA_OK && c[failed] != ctx) return fail(ctx, st, "%s", c[failed]->err.c_str());
    return st;
}

// ---------------------------------------------------------------------------
// host preprocessing shared with the server (koma_server.cpp)
// ---------------------------------------------------------------------------
namespace koma {

int host_phantom32(int64_t n, const double* x, const double* y, const double* z, const double* pd,
                   const double* t1, const double* t2, const double* dw, std::vector<float>& h32, int64_t& n_pad,
                   double (&max_abs)[4], std::string& err) {
    if (n < 0) {
        err = "phantom: n < 0";
        return KOMA_E_INVALID;
    }
    if (n > 0 && (!x || !y || !z || !pd || !t1 || !t2 || !dw)) {
        err = "phantom: NULL array";
        return KOMA_E_INVALID;
    }
    if (!check_spin_values(n, x, y, z, pd, t1, t2, dw, err)) return KOMA_E_INVALID;
    n_pad = std::max<int64_t>(32, (n + 31) / 32 * 32);
    h32.assign(static_cast<size_t>(P32_N * n_pad), 0.f);
    for (int d = 0; d < 4; ++d) max_abs[d] = 0.0;
    const int64_t np = n_pad;
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t j = lo; j < hi; ++j) {
            const double f = dw[j] / (2.0 * kPi);
            split(x[j], &h32[P32_XH * np + j], &h32[P32_XL * np + j]);
            split(y[j], &h32[P32_YH * np + j], &h32[P32_YL * np + j]);
            split(z[j], &h32[P32_ZH * np + j], &h32[P32_ZL * np + j]);
            split(f, &h32[P32_FH * np + j], &h32[P32_FL * np + j]);
            h32[P32_M0 * np + j] = static_cast<float>(pd[j]);
            h32[P32_R1 * np + j] = static_cast<float>(kLog2e / t1[j]);
            h32[P32_R2 * np + j] = static_cast<float>(kLog2e / t2[j]);
        }
    });
    for (int64_t j = 0; j < n; ++j) {
        max_abs[0] = std::max(max_abs[0], std::fabs(x[j]));
        max_abs[1] = std::max(max_abs[1], std::fabs(y[j]));
        max_abs[2] = std::max(max_abs[2], std::fabs(z[j]));
        max_abs[3] = std::max(max_abs[3], std::fabs(dw[j]) / (2.0 * kPi));
    }
    return KOMA_OK;
}

size_t compact_records32_into(const std::vector<Rec32>& r32, Rec32* out) {
    return compact_records32_into(r32.data(), r32.size(), out);
}

size_t compact_records32_into(const Rec32* r32, size_t n_rec, Rec32* out) {
    size_t n = 0;
    for (size_t i = 0; i < n_rec; ++n) {
        const Rec32& q = r32[i];
        if (q.type == REC_RF && q.count > 0 && q.k0 > 0) {
            Rec32 m{};
            m.type = REC_MAP;
            m.count = q.count;
            m.k0 = q.k0 - 1;
            if (out) out[n] = m;
            i += static_cast<size_t>(q.count);
        } else {
            if (out) out[n] = q;
            ++i;
        }
    }
    return n;
}

void compact_records32(const std::vector<Rec32>& r32, std::vector<Rec32>& out) {
    out.resize(compact_records32_into(r32, nullptr));
    compact_records32_into(r32, out.data());
}

int host_check_phantom(int64_t n, const double* x, const double* y, const double* z, const double* pd,
                       const double* t1, const double* t2, const double* dw, std::string& err) {
    if (n < 0) {
        err = "phantom: n < 0";
        return KOMA_E_INVALID;
    }
    if (n > 0 && (!x || !y || !z || !pd || !t1 || !t2 || !dw)) {
        err = "phantom: NULL array";
        return KOMA_E_INVALID;
    }
    return check_spin_values(n, x, y, z, pd, t1, t2, dw, err) ? KOMA_OK : KOMA_E_INVALID;
}

int host_check_sequence(int64_t n_steps, const double* dt, const double* gx, const double* gy, const double* gz,
                        const double* b1_re, const double* b1_im, const uint8_t* adc, koma_sequence_info& info,
                        std::string& err) {
    char buf[160];
    if (n_steps < 0 || !gx || !gy || !gz || !adc || (n_steps > 0 && (!dt || !b1_re || !b1_im))) {
        err = "sequence: n_steps < 0 or a NULL array";
        return KOMA_E_INVALID;
    }
    int64_t count = 0;
    for (int64_t i = 0; i <= n_steps; ++i) {
        if (!std::isfinite(gx[i]) || !std::isfinite(gy[i]) || !std::isfinite(gz[i]) || adc[i] > 1) {
            snprintf(buf, sizeof(buf), "sequence: bad gradient or adc value at time point %lld", static_cast<long long>(i));
            err = buf;
            return KOMA_E_INVALID;
        }
        count += adc[i];
    }
    int64_t n_rf = 0, rf_runs = 0;
    bool prev_rf = false;
    for (int64_t k = 0; k < n_steps; ++k) {
        if (!std::isfinite(dt[k]) || !(dt[k] > 0) || !std::isfinite(b1_re[k]) || !std::isfinite(b1_im[k])) {
            snprintf(buf, sizeof(buf), "sequence: bad dt or B1 at step %lld", static_cast<long long>(k));
            err = buf;
            return KOMA_E_INVALID;
        }
        const bool rf = b1_re[k] != 0.0 || b1_im[k] != 0.0;
        n_rf += rf;
        rf_runs += rf && !prev_rf;
        prev_rf = rf;
    }
    info = koma_sequence_info{};
    info.n_steps = n_steps;
    info.n_adc = count;
    info.n_rf = n_rf;
    info.n_materialize = rf_runs;
    return KOMA_OK;
}

void host_rf_maps32(std::vector<Rec32>& r32, std::vector<RfMapPulse>& pulses, koma_sequence_info& info) {
    RfMapPlan fp;
    plan_rf_maps(r32, fp);
    pulses = fp.pulses;
    info.n_rf_maps = static_cast<int64_t>(fp.pulses.size());
    info.n_rf_map_runs = fp.runs;
    info.n_rf_map_steps = fp.steps;
    info.n_rf_map_pulse_steps = fp.pulse_steps;
}

SerialHostScope::SerialHostScope() : prev(t_host_parallel) { t_host_parallel = false; }
SerialHostScope::~SerialHostScope() { t_host_parallel = prev; }

koma_status sequence_upload_fp32(koma_ctx* ctx, int64_t n_steps, const double* dt, const double* gx,
                                 const double* gy, const double* gz, const double* b1_re, const double* b1_im,
                                 const uint8_t* adc, koma_sequence** out) {
    NvtxRange nvtx_("sequence_upload_fp32");
    return sequence_upload_impl(ctx, n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, false, false, out);
}

int phantom_from_device(koma_ctx* ctx, int64_t n, double* p64, float* p32, const double (&max_abs)[4],
                        double max_pd, const int64_t* group_offsets, int64_t n_groups, bool uni_relax,
                        koma_phantom** out) {
    *out = nullptr;
    if (!ctx || n < 0 || (n > 0 && (!p64 || !p32))) return KOMA_E_INVALID;
    koma_phantom* ph = new (std::nothrow) koma_phantom();
    if (!ph) return KOMA_E_NOMEM;
    ph->ctx = ctx;
    ph->n = n;
    ph->n_pad = std::max<int64_t>(32, (n + 31) / 32 * 32);
    ph->n_groups = group_offsets ? n_groups : 1;
    if (group_offsets) ph->group_offsets.assign(group_offsets, group_offsets + n_groups + 1);
    ph->uni_relax = group_offsets && uni_relax;
    ph->p64 = p64;
    ph->p32 = p32;
    ph->borrowed = true;
    for (int d = 0; d < 4; ++d) ph->max_abs[d] = max_abs[d];
    ph->max_pd = max_pd;
    ctx->live_objects++;
    *out = ph;
    return KOMA_OK;
}

void phantom_free_on(koma_phantom* ph, void* stream) {
    if (!ph) return;
    koma_ctx* ctx = ph->ctx;
    DeviceGuard g(ctx->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!ph->borrowed) {
        dev_free_on(ctx, ph->p32, static_cast<size_t>(P32_N * ph->n_pad) * sizeof(float), st);
        dev_free_on(ctx, ph->p64, static_cast<size_t>(P64_N * ph->n_pad) * sizeof(double), st);
    }
    dev_free_on(ctx, ph->d_cta_begin, ph->table_bytes, st);
    dev_free_on(ctx, ph->d_items, ph->items_bytes, st);
    dev_free_on(ctx, ph->pv32, static_cast<size_t>(PV32_N * ph->n_pad) * sizeof(float), st);
    dev_free_on(ctx, ph->pv64, static_cast<size_t>(3 * ph->n_pad) * sizeof(double), st);
    ctx->live_objects--;
    delete ph;
}

void sequence_free_on(koma_sequence* seq, void* stream) {
    if (!seq) return;
    koma_ctx* ctx = seq->ctx;
    DeviceGuard g(ctx->device);
    dev_free_on(ctx, seq->r32, seq->bytes, static_cast<cudaStream_t>(stream));
    ctx->live_objects--;
    delete seq;
}

int host_records32(int64_t n_steps, const double* dt, const double* gx, const double* gy, const double* gz,
                   const double* b1_re, const double* b1_im, const uint8_t* adc, std::vector<Rec32>& r32,
                   koma_sequence_info& info, std::string& err) {
    RecordBuilder rb;
    rb.reset(false, false);  // the FP32 stream only
    koma_status st = build_records(n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, rb, info, err);
    if (st != KOMA_OK) return st;
    r32.swap(rb.r32);
    return KOMA_OK;
}

}  // namespace koma
