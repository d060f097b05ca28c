// Continuous-batching simulation server (native runtime of libkoma).
//
// Requests (a phantom and a sequence, host arrays) are validated and
// preprocessed on the submitting thread. Grouped requests and requests that
// fill the GPU alone (at least plain_spins spins) go to the second lane: a
// thread of their own that uploads them into a context of the server and
// runs koma_simulate on its stream, one at a time, overlapping the shared
// launches below. For the others, one worker thread:
//   * admits them in arrival order while the device-memory budget allows
//     (stream-ordered allocations from a server-owned pool, so a finishing
//     request frees its memory without a device-wide synchronisation);
//   * keeps two launches of the serving kernel (K4) in flight on two streams;
//     each launch takes CTA-batches (512 spins of one request) from every
//     admitted request, shortest remaining work first, enough to fill the GPU
//     and up to a work cap, so a request arriving while others run joins the
//     next launch and shares it with them;
//   * when all batches of a request are done, reduces its partial rows in a
//     fixed order (K2), copies the signal to pinned host memory and frees
//     the request's device memory.
// A request's decomposition into batches does not depend on the other
// requests, so its result is bitwise the same alone and in any mix.
// Each slot's launch is a CUDA graph (copy of the batch table, including the
// zeroed batch counter, then K4); only the copy's length changes per launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "koma.h"
#include "koma_internal.h"
#include "koma_host.h"

namespace {

constexpr int kBlock = 128;                        // K4 CTA: 4 warps
constexpr int kWarps = kBlock / 32;
constexpr int64_t kBatchSpins = kWarps * 32 * 4;   // 4 spins per thread
constexpr int kSlots = 2;
constexpr int kLanes = 4;                          // threads (contexts, streams) of the second lane
// requests this large take the second lane: only those that fill the GPU
// alone (on the 2,000-request serving mix 2^19 served 1.63-1.79e12 spin-steps/s
// saturated against 1.40-1.51e12 at 2^15, p99 55-59 against 52-54 ms)
constexpr int64_t kDefaultPlainSpins = 524288;
constexpr size_t kHeader = 16;                     // int64 n_batches, int32 counter, int32 status
constexpr size_t kStatusOff = 12;                  // the launch's device status word in the header

enum ReqState { PENDING, ADMITTED, LANE, REDUCING, DONE, FAILED };

struct Req {
    uint64_t id = 0;
    double t_submit = 0, t_admit = -1, t_done = -1;
    int64_t n = 0, n_pad = 0, n_steps = 0, n_adc = 0, n_rec = 0, n_adc_runs = 0;
    std::vector<float> h32;
    std::vector<koma::Rec32> recs;
    double max_abs[4] = {0, 0, 0, 0};
    float ext[4] = {0, 0, 0, 0};
    int used = 0;
    double work_per_spin = 0;  // relative cost units per spin (RF step = 1)
    int64_t n_batches = 0;
    // the record stream is walked in chunks of `chunk` records (checkpointed
    // between launches); a unit of work = one batch x one chunk
    int64_t chunk = 0, n_chunks = 1, units_total = 0, units_done = 0;
    std::vector<double> chunk_work;   // work units per spin of each chunk
    std::vector<int64_t> chunk_hdr;   // RF run header a chunk starts inside, or -1
    std::vector<int64_t> chunk_begin; // first record of each chunk, then n_rec
    // repeated RF pulses: one map per slot, computed per spin at admission
    // from the full record stream; `recs` is then the compacted stream
    std::vector<koma::RfMapPulse> pulses;
    std::vector<koma::Rec32> recs_full;
    float* dmaps = nullptr;
    koma::RfMapPulse* dpulses = nullptr;
    koma::Rec32* drec_full = nullptr;
    std::vector<int32_t> batch_next;  // next chunk of each batch
    std::vector<char> batch_busy;     // batch is in a launch in flight
    double rem_work = 0;
    float* dstate = nullptr;
    int launches = 0;
    size_t dev_bytes = 0;
    float* d32 = nullptr;
    koma::Rec32* drec = nullptr;
    float2* drows = nullptr;
    double* dsig = nullptr;
    double* hsig = nullptr;  // pinned, from the server's pool (size class hsig_cls)
    int hsig_cls = -1;
    cudaEvent_t ev_up = nullptr, ev_done = nullptr;
    ReqState state = PENDING;
    koma_status err = KOMA_OK;
    std::string msg;
    bool retired = false;  // out of the worker's lists: the waiter may delete it
    double prep_s = 0, upload_s = 0, run_s = 0;  // host time of submit, lane upload, lane run
    // second lane (koma_simulate): the host arrays until the upload
    bool lane = false;
    int64_t n_groups = 1;
    std::unique_ptr<double[]> ph64;   // x, y, z, pd, t1, t2, dw, each n long (host path only)
    // device path: the phantom uploaded, checked and converted at submit
    // (blocks from the server's pool, counted in `used` until retirement)
    double* dp64 = nullptr;
    float* dp32 = nullptr;
    size_t ph_dev_bytes = 0;
    double max_pd = 0;
    bool uni_relax = false;
    std::vector<int64_t> offsets;     // group offsets (grouped requests)
    std::vector<double> sq64;         // dt [n_steps], gx, gy, gz [n_steps + 1], b1 re, im [n_steps]
    std::vector<uint8_t> sq_adc;

    // uploaded by the submitting thread (its device memory already counted)
    bool uploaded = false;

    double remaining_work() const { return rem_work; }
};

struct Slot {
    cudaStream_t st = nullptr;
    char* h_buf = nullptr;  // pinned: header + BatchDesc[cap]
    char* d_buf = nullptr;
    int64_t cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<std::pair<Req*, int32_t>> members;  // (request, batch) per table entry
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct koma_server {
    int device = 0;
    int64_t chunk = 4096;  // records per chunk of a batch's walk
    int64_t plain_spins = kDefaultPlainSpins;  // requests this large run in the second lane (<= 0: never)
    // the second lane: kLanes threads, each with a context and a stream of
    // its own, so one request's upload overlaps another's kernels and
    // requests that do not fill the GPU run side by side
    koma_ctx* lane_ctx[kLanes] = {};
    cudaStream_t s_lane[kLanes] = {};
    std::thread lane_worker[kLanes];
    std::deque<Req*> lane_q;
    std::condition_variable cv_lane;
    int64_t lane_runs = 0;
    // streams (with a conversion status word each) for the uploads that
    // submit calls do on their own threads
    struct UpSlot {
        cudaStream_t st = nullptr;
        koma::ConvertStatus* d_cs = nullptr;
        koma::ConvertStatus* h_cs = nullptr;  // pinned
    };
    std::mutex up_mu;
    std::vector<UpSlot*> up_free, up_all;
    // pinned result buffers, reused: free lists by power-of-two size class
    // (cudaMallocHost / cudaFreeHost per request cost driver time, and a
    // free waits for the device)
    std::mutex host_mu;
    std::vector<void*> host_free[48];
    size_t budget = 0, used = 0, peak = 0;
    int max_active = 64;
    double launch_work = 0;  // work units per launch (cap)
    int sm_count = 0, grid = 0;
    double t0 = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    std::deque<Req*> pending;
    std::vector<Req*> active;
    std::map<uint64_t, Req*> all;
    uint64_t next_id = 1;
    cudaStream_t s_up = nullptr, s_red = nullptr;
    cudaMemPool_t pool = nullptr;
    Slot slots[kSlots];
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, launches = 0, batches = 0;
    std::string fatal;
};

namespace {

// NVTX range for the scope (a no-op unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

koma_status cuda_err(koma_server* S, cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    S->fatal = buf;
    return e == cudaErrorMemoryAllocation ? KOMA_E_NOMEM : KOMA_E_CUDA;
}

// A pinned host buffer of at least `bytes` (4 KiB and up, power-of-two
// classes) from the server's pool; *cls receives its class. Null on failure.
double* host_acquire(koma_server* S, size_t bytes, int* cls) {
    *cls = -1;
    if (bytes > (size_t{1} << 47)) return nullptr;
    int c = 12;
    while ((size_t{1} << c) < bytes) ++c;
    *cls = c;
    {
        std::lock_guard<std::mutex> lk(S->host_mu);
        if (!S->host_free[c].empty()) {
            void* p = S->host_free[c].back();
            S->host_free[c].pop_back();
            return static_cast<double*>(p);
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, size_t{1} << c) != cudaSuccess) {
        cudaGetLastError();
        *cls = -1;
        return nullptr;
    }
    return static_cast<double*>(p);
}

// Back to the pool (only once nothing copies into it any more).
void host_release(koma_server* S, Req* r) {
    if (!r->hsig) return;
    {
        std::lock_guard<std::mutex> lk(S->host_mu);
        S->host_free[r->hsig_cls].push_back(r->hsig);
    }
    r->hsig = nullptr;
    r->hsig_cls = -1;
}

// An upload stream (with its conversion status word) for a submitting
// thread: a free one, else a new one; null if none can be made.
koma_server::UpSlot* up_acquire(koma_server* S) {
    {
        std::lock_guard<std::mutex> lk(S->up_mu);
        if (!S->up_free.empty()) {
            koma_server::UpSlot* U = S->up_free.back();
            S->up_free.pop_back();
            return U;
        }
    }
    koma_server::UpSlot* U = new (std::nothrow) koma_server::UpSlot();
    if (!U) return nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&U->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&U->d_cs), sizeof(koma::ConvertStatus));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&U->h_cs), sizeof(koma::ConvertStatus));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (U->h_cs) cudaFreeHost(U->h_cs);
        if (U->d_cs) cudaFree(U->d_cs);
        if (U->st) cudaStreamDestroy(U->st);
        delete U;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(S->up_mu);
    S->up_all.push_back(U);
    return U;
}

void up_release(koma_server* S, koma_server::UpSlot* U) {
    if (!U) return;
    std::lock_guard<std::mutex> lk(S->up_mu);
    S->up_free.push_back(U);
}

// A large request's phantom on the device, done by the submitting thread:
// the caller's rows are copied into blocks of the server's pool on one of
// the upload streams, and the conversion kernel checks every spin, takes the
// extents and builds the FP32 block (what koma_phantom_upload does); the
// lane later simulates on these blocks without a host copy or a second
// upload. KOMA_E_INVALID (err set) for invalid spins; KOMA_E_NOMEM when the
// budget or the pool has no room (the caller then keeps a host copy).
koma_status upload_lane_phantom(koma_server* S, Req* r, int64_t n, const double* x, const double* y,
                                const double* z, const double* pd, const double* t1, const double* t2,
                                const double* dw, std::string& err) {
    const int64_t np = r->n_pad;
    const size_t b64 = static_cast<size_t>(koma::P64_N * np) * sizeof(double),
                 b32 = static_cast<size_t>(koma::P32_N * np) * sizeof(float);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->budget && S->used + b64 + b32 > S->budget) return KOMA_E_NOMEM;
        S->used += b64 + b32;
        S->peak = std::max(S->peak, S->used);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->device) cudaSetDevice(S->device);
    koma_server::UpSlot* U = up_acquire(S);
    cudaError_t e = U ? cudaSuccess : cudaErrorMemoryAllocation;
    double* p64 = nullptr;
    float* p32 = nullptr;
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&p64), b64, S->pool, U->st);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&p32), b32, S->pool, U->st);
    const double* rows[koma::P64_N] = {x, y, z, dw, t1, t2, pd};  // the order of enum P64
    for (int k = 0; k < koma::P64_N && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(p64 + k * np, rows[k], static_cast<size_t>(n) * sizeof(double), cudaMemcpyHostToDevice,
                            U->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(U->d_cs, 0, sizeof(koma::ConvertStatus), U->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&U->d_cs->first_bad, 0xff, sizeof(unsigned long long), U->st);
    if (e == cudaSuccess) e = static_cast<cudaError_t>(koma::launch_phantom_convert(p64, p32, n, np, U->d_cs, U->st));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(U->h_cs, U->d_cs, sizeof(koma::ConvertStatus), cudaMemcpyDeviceToHost, U->st);
    if (U) {
        const cudaError_t es = cudaStreamSynchronize(U->st);
        if (e == cudaSuccess) e = es;
    }
    koma_status st = KOMA_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        st = e == cudaErrorMemoryAllocation ? KOMA_E_NOMEM : KOMA_E_CUDA;
        err = std::string("server_submit: phantom upload: ") + cudaGetErrorString(e);
    } else if (U->h_cs->first_bad != ~0ull) {
        st = static_cast<koma_status>(koma::host_check_phantom(n, x, y, z, pd, t1, t2, dw, err));
        if (st == KOMA_OK) {  // the device found what the host check did not: report the index
            st = KOMA_E_INVALID;
            err = "phantom: invalid spin " + std::to_string(U->h_cs->first_bad);
        }
    } else {
        for (int d = 0; d < 4; ++d) std::memcpy(&r->max_abs[d], &U->h_cs->max_bits[d], sizeof(double));
        std::memcpy(&r->max_pd, &U->h_cs->max_bits[4], sizeof(double));
        r->dp64 = p64;
        r->dp32 = p32;
        r->ph_dev_bytes = b64 + b32;
    }
    if (st != KOMA_OK) {
        if (U) {
            if (p64) cudaFreeAsync(p64, U->st);
            if (p32) cudaFreeAsync(p32, U->st);
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->used -= std::min(S->used, b64 + b32);
    }
    up_release(S, U);
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    return st;
}

size_t map_bytes(const Req* r) {
    return r->pulses.size() * koma::kRfMapFloats * static_cast<size_t>(r->n_pad) * sizeof(float);
}

size_t req_bytes(const Req* r) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    if (r->lane) {
        // koma_simulate lane: FP32 and FP64 phantom blocks, three record
        // streams, per-CTA partial rows (at most a few thousand CTAs), the
        // readout's snapshots (bounded by one row per ADC run) and the maps
        const size_t np = static_cast<size_t>(r->n_pad);
        // (the phantom blocks of a request uploaded at submit are counted there)
        return (r->dp64 ? 0 : np * (koma::P32_N * sizeof(float) + koma::P64_N * sizeof(double))) +
               static_cast<size_t>(r->n_rec) * 3 * sizeof(koma::Rec64) +
               static_cast<size_t>(r->n_groups) * static_cast<size_t>(r->n_adc) * 16 +
               static_cast<size_t>(4096) * static_cast<size_t>(r->n_adc) * sizeof(float2) +
               static_cast<size_t>(r->n_adc_runs) * np * sizeof(float2) + map_bytes(r) + (size_t{1} << 20);
    }
    return al(r->h32.size() * sizeof(float)) + al(r->recs.size() * sizeof(koma::Rec32)) +
           al(static_cast<size_t>(r->n_batches) * kWarps * r->n_adc * sizeof(float2)) +
           al(static_cast<size_t>(r->n_adc) * 2 * sizeof(double)) +
           (r->n_chunks > 1 ? al(static_cast<size_t>(3 * r->n_pad) * sizeof(float)) : 0) +
           (r->pulses.empty() ? 0 : al(map_bytes(r)) + al(r->pulses.size() * sizeof(koma::RfMapPulse)) +
                                        al(r->recs_full.size() * sizeof(koma::Rec32)));
}

void fail_req(Req* r, koma_status st, const std::string& m) {
    r->state = FAILED;
    r->err = st;
    r->msg = m;
}

// Allocate and upload a request of the shared lane on stream `st` (the
// submitting thread's upload stream, or the worker's s_up): device blocks
// from the server's pool, the copies, the maps of its repeated pulses; ev_up
// marks the end. Nothing here waits for the copies.
koma_status admit(koma_server* S, Req* r, cudaStream_t st) {
    NvtxRange nvtx_("server admit");
    const size_t b32 = r->h32.size() * sizeof(float), brec = r->recs.size() * sizeof(koma::Rec32);
    const size_t brows = static_cast<size_t>(r->n_batches) * kWarps * r->n_adc * sizeof(float2);
    const size_t bsig = static_cast<size_t>(r->n_adc) * 2 * sizeof(double);
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->d32), b32, S->pool, st);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->drec), brec, S->pool, st);
    if (e == cudaSuccess && brows)
        e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->drows), brows, S->pool, st);
    if (e == cudaSuccess && bsig) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->dsig), bsig, S->pool, st);
    if (e == cudaSuccess && bsig) {
        r->hsig = host_acquire(S, bsig, &r->hsig_cls);
        if (!r->hsig) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess && r->n_chunks > 1)
        e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->dstate), static_cast<size_t>(3 * r->n_pad) * sizeof(float),
                                    S->pool, st);
    if (e == cudaSuccess && !r->pulses.empty() && r->n > 0) {
        e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->dmaps), map_bytes(r), S->pool, st);
        if (e == cudaSuccess)
            e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->dpulses),
                                        r->pulses.size() * sizeof(koma::RfMapPulse), S->pool, st);
        if (e == cudaSuccess)
            e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->drec_full),
                                        r->recs_full.size() * sizeof(koma::Rec32), S->pool, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->d32, r->h32.data(), b32, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && brec)
        e = cudaMemcpyAsync(r->drec, r->recs.data(), brec, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r->dmaps) {
        // the maps of the request's repeated pulses, before its first launch
        e = cudaMemcpyAsync(r->dpulses, r->pulses.data(), r->pulses.size() * sizeof(koma::RfMapPulse),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->drec_full, r->recs_full.data(), r->recs_full.size() * sizeof(koma::Rec32),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            koma::RfMapArgs F;
            F.p32 = r->d32;
            F.n_pad = r->n_pad;
            F.n = r->n;
            F.rec = r->drec_full;
            F.pulses = r->dpulses;
            F.n_pulses = static_cast<int>(r->pulses.size());
            F.maps = r->dmaps;
            for (int d = 0; d < 4; ++d) F.ext[d] = r->ext[d];
            e = static_cast<cudaError_t>(koma::launch_rf_maps(F, st));
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_up, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev_up, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? KOMA_E_NOMEM : KOMA_E_CUDA;
    r->dev_bytes = req_bytes(r);
    r->t_admit = now_s();
    r->state = ADMITTED;
    return KOMA_OK;
}

// The request's device blocks of the shared lane, freed in order on `st`.
void free_shared_blocks(Req* r, cudaStream_t st) {
    for (void** p : {reinterpret_cast<void**>(&r->d32), reinterpret_cast<void**>(&r->drec),
                     reinterpret_cast<void**>(&r->drows), reinterpret_cast<void**>(&r->dsig),
                     reinterpret_cast<void**>(&r->dstate), reinterpret_cast<void**>(&r->dmaps),
                     reinterpret_cast<void**>(&r->dpulses), reinterpret_cast<void**>(&r->drec_full)}) {
        if (*p) cudaFreeAsync(*p, st);
        *p = nullptr;
    }
}

void release_device(koma_server* S, Req* r) {
    if (r->dp64) cudaFreeAsync(r->dp64, S->s_red);
    if (r->dp32) cudaFreeAsync(r->dp32, S->s_red);
    r->dp64 = nullptr;
    r->dp32 = nullptr;
    S->used -= std::min(S->used, r->ph_dev_bytes);
    r->ph_dev_bytes = 0;
    free_shared_blocks(r, S->s_red);
    r->recs_full.clear();
    r->recs_full.shrink_to_fit();
    S->used -= std::min(S->used, r->dev_bytes);
    r->dev_bytes = 0;
    r->h32.clear();
    r->h32.shrink_to_fit();
    r->recs.clear();
    r->recs.shrink_to_fit();
}

// A request of the shared lane uploaded by the submitting thread when the
// memory budget has room for it now: the allocations, copies and map
// pre-pass go on an upload stream (ev_up orders its launches after them),
// and the host arrays are released at once. Otherwise, or if an allocation
// fails, the worker uploads it at admission.
void upload_shared_request(koma_server* S, Req* r) {
    const size_t need = req_bytes(r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop || (S->budget && S->used + need > S->budget)) return;
        S->used += need;
        S->peak = std::max(S->peak, S->used);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->device) cudaSetDevice(S->device);
    koma_server::UpSlot* U = up_acquire(S);
    const koma_status st = U ? admit(S, r, U->st) : KOMA_E_NOMEM;
    if (st == KOMA_OK) {
        r->uploaded = true;  // r->dev_bytes == need: admit counted the same arrays
        std::vector<float>().swap(r->h32);
        std::vector<koma::Rec32>().swap(r->recs);
        std::vector<koma::Rec32>().swap(r->recs_full);
    } else {
        cudaGetLastError();
        if (U) cudaStreamSynchronize(U->st);  // nothing may still copy into the blocks
        free_shared_blocks(r, U ? U->st : S->s_red);
        host_release(S, r);
        if (r->ev_up) cudaEventDestroy(r->ev_up);
        if (r->ev_done) cudaEventDestroy(r->ev_done);
        r->ev_up = r->ev_done = nullptr;
        r->dev_bytes = 0;
        r->state = PENDING;
        std::lock_guard<std::mutex> lk(S->mu);
        S->used -= std::min(S->used, need);
    }
    up_release(S, U);
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
}

koma_status make_slot(koma_server* S, Slot& sl, int64_t cap) {
    sl.cap = cap;
    const size_t bytes = kHeader + static_cast<size_t>(cap) * sizeof(koma::BatchDesc);
    cudaError_t e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.h_buf), bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.d_buf), bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_err(S, e, "server: slot set-up");
    std::memset(sl.h_buf, 0, bytes);
    // graph: copy (header with zero counter + table) -> serving kernel
    koma::BatchArgs A;
    A.desc = reinterpret_cast<const koma::BatchDesc*>(sl.d_buf + kHeader);
    A.n_batches_dev = reinterpret_cast<const int64_t*>(sl.d_buf);
    A.counter = reinterpret_cast<int*>(sl.d_buf + 8);
    // each launch has its own status word: zeroed by the table copy, read
    // back into the host header after the kernel
    A.status = reinterpret_cast<int*>(sl.d_buf + kStatusOff);
    e = cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemcpyAsync(sl.d_buf, sl.h_buf, kHeader + sizeof(koma::BatchDesc), cudaMemcpyHostToDevice, sl.st);
        koma::launch_batches(A, S->grid, kBlock, sl.st);
        cudaMemcpyAsync(sl.h_buf + kStatusOff, sl.d_buf + kStatusOff, sizeof(int), cudaMemcpyDeviceToHost, sl.st);
        e = cudaStreamEndCapture(sl.st, &sl.graph);
    }
    if (e != cudaSuccess) return cuda_err(S, e, "server: graph capture");
    size_t n_nodes = 0;
    cudaGraphGetNodes(sl.graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    cudaGraphGetNodes(sl.graph, nodes.data(), &n_nodes);
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nd, &t);
        if (t != cudaGraphNodeTypeMemcpy) continue;
        cudaMemcpy3DParms mp{};
        cudaGraphMemcpyNodeGetParams(nd, &mp);
        if (mp.kind == cudaMemcpyHostToDevice) sl.copy = nd;  // the table copy (the other reads the status)
    }
    if (!sl.copy) return cuda_err(S, cudaErrorUnknown, "server: graph has no copy node");
    e = cudaGraphInstantiate(&sl.exec, sl.graph, 0);
    if (e != cudaSuccess) return cuda_err(S, e, "server: graph instantiate");
    return KOMA_OK;
}

// Fill a free slot with units (batch x chunk) and launch it. Requests are
// taken shortest remaining work first; the launch holds at least enough units
// to fill the GPU (when there are that many) and stops at the work cap.
bool launch_slot(koma_server* S, Slot& sl) {
    NvtxRange nvtx_("server launch");
    std::vector<Req*> cand;
    for (Req* r : S->active)
        if (r->state == ADMITTED && r->units_done + 0 < r->units_total) cand.push_back(r);
    if (cand.empty()) return false;
    std::sort(cand.begin(), cand.end(), [](const Req* a, const Req* b) {
        return a->remaining_work() < b->remaining_work() ||
               (a->remaining_work() == b->remaining_work() && a->id < b->id);
    });
    koma::BatchDesc* tab = reinterpret_cast<koma::BatchDesc*>(sl.h_buf + kHeader);
    int64_t nb = 0;
    double work = 0;
    sl.members.clear();
    for (Req* r : cand) {
        bool took = false;
        for (int64_t b = 0; b < r->n_batches && nb < sl.cap; ++b) {
            if (r->batch_busy[b] || r->batch_next[b] >= r->n_chunks) continue;
            const int32_t c = r->batch_next[b];
            const double w = kBatchSpins * r->chunk_work[c];
            if (nb >= S->grid && work + w > S->launch_work) break;
            koma::BatchDesc& D = tab[nb++];
            std::memset(&D, 0, sizeof(D));
            D.p32 = r->d32;
            D.n_pad = r->n_pad;
            D.rec = r->drec;
            D.n_rec = r->n_rec;
            D.rows = r->drows + static_cast<size_t>(b) * kWarps * r->n_adc;
            D.n_adc = r->n_adc;
            D.spin_begin = b * kBatchSpins;
            D.spin_end = std::min(r->n, D.spin_begin + kBatchSpins);
            D.rec_begin = r->chunk_begin[static_cast<size_t>(c)];
            D.rec_end = r->chunk_begin[static_cast<size_t>(c) + 1];
            D.state = r->dstate;
            D.rf_hdr = r->chunk_hdr[c];
            D.rf_maps = r->dmaps;
            D.n_rf_maps = r->dmaps ? static_cast<int>(r->pulses.size()) : 0;
            for (int d = 0; d < 4; ++d) D.ext[d] = r->ext[d];
            D.used = r->used;
            r->batch_busy[b] = 1;
            r->rem_work -= w;
            sl.members.emplace_back(r, static_cast<int32_t>(b));
            work += w;
            took = true;
        }
        if (took) {
            ++r->launches;
            cudaStreamWaitEvent(sl.st, r->ev_up, 0);  // no-op once the upload is done
        }
        if (nb >= sl.cap || (nb >= S->grid && work >= S->launch_work)) break;
    }
    if (nb == 0) return false;
    *reinterpret_cast<int64_t*>(sl.h_buf) = nb;
    *reinterpret_cast<int32_t*>(sl.h_buf + 8) = 0;
    *reinterpret_cast<int32_t*>(sl.h_buf + kStatusOff) = 0;
    cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(sl.exec, sl.copy, sl.d_buf, sl.h_buf,
                                                       kHeader + static_cast<size_t>(nb) * sizeof(koma::BatchDesc),
                                                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, sl.st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.st);
    if (e != cudaSuccess) {
        for (auto& m : sl.members) fail_req(m.first, KOMA_E_CUDA, cudaGetErrorString(e));
        sl.members.clear();
        return false;
    }
    sl.busy = true;
    ++S->launches;
    S->batches += nb;
    return true;
}

void finalize(koma_server* S, Req* r) {
    NvtxRange nvtx_("server finalize");
    koma::ReduceArgs R;
    R.partial = r->drows;
    R.grid = static_cast<int>(r->n_batches * kWarps);
    R.n_groups = 1;
    R.n_adc = r->n_adc;
    R.sig = r->dsig;
    int e = r->n_adc > 0 ? koma::launch_reduce(R, false, S->s_red) : cudaSuccess;
    cudaError_t ce = static_cast<cudaError_t>(e);
    if (ce == cudaSuccess && r->n_adc > 0)
        ce = cudaMemcpyAsync(r->hsig, r->dsig, static_cast<size_t>(r->n_adc) * 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, S->s_red);
    if (ce == cudaSuccess) ce = cudaEventRecord(r->ev_done, S->s_red);
    if (ce != cudaSuccess) {
        fail_req(r, KOMA_E_CUDA, cudaGetErrorString(ce));
        return;
    }
    r->state = REDUCING;
}

void worker_loop(koma_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        // admission (arrival order, device-memory budget)
        while (!S->pending.empty() && static_cast<int>(S->active.size()) < S->max_active) {
            Req* r = S->pending.front();
            if (r->uploaded) {  // its submitting thread uploaded it (memory counted there)
                S->pending.pop_front();
                r->t_admit = now_s();
                S->active.push_back(r);
                if (r->units_total == 0) finalize(S, r);  // nothing to step
                progress = true;
                continue;
            }
            const size_t need = req_bytes(r);
            if (S->budget && S->used + need > S->budget) {
                if (S->active.empty()) {
                    S->pending.pop_front();
                    fail_req(r, KOMA_E_NOMEM, "request needs more device memory than the server's budget");
                    r->t_done = now_s();
                    r->retired = true;
                    S->failed++;
                    S->cv_done.notify_all();
                    progress = true;
                    continue;
                }
                break;
            }
            S->pending.pop_front();
            if (r->lane) {
                // the second lane uploads and runs it (its thread, its stream)
                r->t_admit = now_s();
                r->state = LANE;
                r->dev_bytes = need;
                S->used += need;
                S->peak = std::max(S->peak, S->used);
                S->active.push_back(r);
                S->lane_q.push_back(r);
                S->cv_lane.notify_all();
                progress = true;
                continue;
            }
            const koma_status st = admit(S, r, S->s_up);
            if (st != KOMA_OK) {
                release_device(S, r);
                fail_req(r, st, "admission failed (device allocation or upload)");
                r->t_done = now_s();
                r->retired = true;
                S->failed++;
                S->cv_done.notify_all();
            } else {
                S->used += r->dev_bytes;
                S->peak = std::max(S->peak, S->used);
                S->active.push_back(r);
                if (r->units_total == 0) finalize(S, r);  // nothing to step
            }
            progress = true;
        }
        // completed launches
        for (Slot& sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            sl.busy = false;
            progress = true;
            // the launch's device status: a bounded wait that gave up, or a
            // record the kernel's bounds checks skipped
            const int dev_flag = q == cudaSuccess ? *reinterpret_cast<volatile int32_t*>(sl.h_buf + kStatusOff) : 0;
            for (auto& m : sl.members) {
                Req* r = m.first;
                if (q != cudaSuccess) {
                    fail_req(r, KOMA_E_CUDA, cudaGetErrorString(q));
                    continue;
                }
                if (dev_flag) {
                    if (r->state != FAILED)
                        fail_req(r, (dev_flag & (koma::kStatusTimeout | koma::kStatusWaitCheck)) ? KOMA_E_TIMEOUT : KOMA_E_INTERNAL,
                                 (dev_flag & (koma::kStatusTimeout | koma::kStatusWaitCheck))
                                     ? "serving kernel: a bounded device-side wait gave up"
                                     : "serving kernel: a record pointed outside the request's buffers");
                    continue;
                }
                r->batch_busy[m.second] = 0;
                ++r->batch_next[m.second];
                ++r->units_done;
                if (r->state == ADMITTED && r->units_done == r->units_total) finalize(S, r);
            }
            sl.members.clear();
        }
        // new launches
        for (Slot& sl : S->slots)
            if (!sl.busy && launch_slot(S, sl)) progress = true;
        // finished requests
        for (size_t i = 0; i < S->active.size();) {
            Req* r = S->active[i];
            bool out = false;
            if (r->lane && r->state == DONE) {
                S->completed++;  // the second lane finished it
                out = true;
            } else if (r->state == REDUCING) {
                const cudaError_t q = cudaEventQuery(r->ev_done);
                if (q != cudaErrorNotReady) {
                    if (q == cudaSuccess) {
                        r->state = DONE;
                        S->completed++;
                    } else {
                        fail_req(r, KOMA_E_CUDA, cudaGetErrorString(q));
                        S->failed++;
                    }
                    r->t_done = now_s();
                    out = true;
                }
            } else if (r->state == FAILED) {
                // wait until no launch still uses its memory
                bool in_use = false;
                for (Slot& sl : S->slots)
                    for (auto& m : sl.members) in_use |= m.first == r;
                if (!in_use) {
                    if (r->t_done < 0) r->t_done = now_s();
                    S->failed++;
                    out = true;
                }
            }
            if (out) {
                release_device(S, r);
                r->retired = true;
                S->active.erase(S->active.begin() + static_cast<long>(i));
                S->cv_done.notify_all();
                progress = true;
            } else {
                ++i;
            }
        }
        const bool idle = S->pending.empty() && S->active.empty();
        if (S->stop && idle) break;
        if (idle) {
            S->cv_work.wait(lk);
        } else if (!progress) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

// Second lane, thread k: grouped requests and large requests through the
// koma_simulate path (uploads, maps of repeated pulses, the Bloch or grouped
// kernel, the tensor-core readout, the reduction) on the thread's own
// context and stream, overlapping the other lane threads and the shared
// launches of the worker. The result goes to the request's pinned buffer;
// the worker retires the request.
void lane_loop(koma_server* S, int k) {
    cudaSetDevice(S->device);
    const koma::SerialHostScope serial_;  // the lanes run side by side: no worker pool
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_lane.wait(lk, [&] { return S->stop || !S->lane_q.empty(); });
        if (S->lane_q.empty()) {
            if (S->stop) break;
            continue;
        }
        Req* r = S->lane_q.front();
        S->lane_q.pop_front();
        lk.unlock();
        NvtxRange nvtx_("server lane run");
        koma_ctx* ctx = S->lane_ctx[k];
        cudaStream_t st_k = S->s_lane[k];
        const int64_t n = r->n, ns = r->n_steps;
        const double* P = r->ph64.get();
        const double* Q = r->sq64.data();
        koma_phantom* ph = nullptr;
        koma_sequence* seq = nullptr;
        const double t_up = now_s();
        const int64_t* offs = r->n_groups > 1 ? r->offsets.data() : nullptr;
        koma_status st = r->dp64 ? static_cast<koma_status>(koma::phantom_from_device(
                                       ctx, n, r->dp64, r->dp32, r->max_abs, r->max_pd, offs, r->n_groups,
                                       r->uni_relax, &ph))
                                 : koma_phantom_upload(ctx, n, P, P + n, P + 2 * n, P + 3 * n, P + 4 * n,
                                                       P + 5 * n, P + 6 * n, offs, r->n_groups, &ph);
        if (st == KOMA_OK)
            st = koma::sequence_upload_fp32(ctx, ns, Q, Q + ns, Q + 2 * ns + 1, Q + 3 * ns + 2, Q + 4 * ns + 3,
                                            Q + 5 * ns + 3, r->sq_adc.data(), &seq);
        const double t_run = now_s();
        const size_t out_bytes = static_cast<size_t>(r->n_groups * r->n_adc) * 2 * sizeof(double);
        double* dsig = nullptr;
        cudaError_t e = cudaSuccess;
        if (st == KOMA_OK && out_bytes) {
            e = cudaMallocAsync(reinterpret_cast<void**>(&dsig), out_bytes, st_k);
            if (e == cudaSuccess) {
                r->hsig = host_acquire(S, out_bytes, &r->hsig_cls);
                if (!r->hsig) e = cudaErrorMemoryAllocation;
            }
            if (e != cudaSuccess) st = KOMA_E_NOMEM;
        }
        if (st == KOMA_OK) st = koma_simulate(ctx, ph, seq, KOMA_FP32_SPLITPHASE, dsig, st_k);
        if (st == KOMA_OK && out_bytes)
            e = cudaMemcpyAsync(r->hsig, dsig, out_bytes, cudaMemcpyDeviceToHost, st_k);
        if (st == KOMA_OK && e == cudaSuccess) st = koma_sync(ctx, st_k);
        else if (st == KOMA_OK) st = KOMA_E_CUDA;
        std::string msg = st != KOMA_OK ? std::string(koma_last_error(ctx)) : std::string();
        // every use of these was on st_k: frees ordered there, no device-wide wait
        if (dsig) cudaFreeAsync(dsig, st_k);
        koma::sequence_free_on(seq, st_k);
        koma::phantom_free_on(ph, st_k);
        cudaStreamSynchronize(st_k);  // also after a failed launch: nothing may still read the blocks
        const double t_end = now_s();
        lk.lock();
        r->upload_s = t_run - t_up;
        r->run_s = t_end - t_run;
        r->ph64.reset();
        r->sq64.clear();
        r->sq64.shrink_to_fit();
        r->sq_adc.clear();
        r->sq_adc.shrink_to_fit();
        r->launches = 1;
        S->lane_runs++;
        if (st == KOMA_OK) {
            r->state = DONE;
        } else {
            char shape[128];
            snprintf(shape, sizeof(shape), " (request of %lld spins, %lld steps, %lld samples)",
                     static_cast<long long>(r->n), static_cast<long long>(r->n_steps),
                     static_cast<long long>(r->n_adc));
            fail_req(r, st, (msg.empty() ? std::string("second lane: simulation failed") : msg) + shape);
        }
        r->t_done = now_s();
    }
}

}  // namespace

extern "C" koma_status koma_server_create(const koma_server_config* cfg, koma_server** out) {
    if (!out) return KOMA_E_INVALID;
    *out = nullptr;
    koma_server_config c{};
    if (cfg) c = *cfg;
    if (c.device < 0 || c.max_active < 0 || c.launch_work < 0) return KOMA_E_INVALID;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || c.device >= count) {
        cudaGetLastError();
        return KOMA_E_CUDA;
    }
    koma_server* S = new (std::nothrow) koma_server();
    if (!S) return KOMA_E_NOMEM;
    S->device = c.device;
    S->budget = c.mem_budget_bytes;
    S->max_active = c.max_active > 0 ? c.max_active : 64;
    // default cap: ~4 ms of the serving kernel at ~4.5e11 RF spin-steps/s
    S->launch_work = c.launch_work > 0 ? c.launch_work : 1.8e9;
    if (c.chunk_records > 0) S->chunk = c.chunk_records;
    if (c.plain_spins != 0) S->plain_spins = c.plain_spins;
    S->t0 = now_s();
    int prev = -1;
    cudaGetDevice(&prev);
    koma_status st = KOMA_OK;
    cudaError_t e = cudaSetDevice(S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_red, cudaStreamNonBlocking);
    for (int k = 0; k < kLanes && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&S->s_lane[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        e = cudaMemPoolCreate(&S->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = ~0ull;  // keep freed memory in the pool for reuse
            cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e != cudaSuccess) st = cuda_err(S, e, "server: set-up");
    for (int k = 0; k < kLanes && st == KOMA_OK; ++k) st = koma_init(S->device, 0, &S->lane_ctx[k]);
    if (st == KOMA_OK) {
        const int per_sm = std::max(1, koma::batches_ctas_per_sm(kBlock));
        S->grid = S->sm_count * per_sm;
        for (Slot& sl : S->slots) {
            st = make_slot(S, sl, std::max<int64_t>(4096, 4 * S->grid));
            if (st != KOMA_OK) break;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st != KOMA_OK) {
        koma_server_destroy(S);
        return st;
    }
    S->worker = std::thread(worker_loop, S);
    for (int k = 0; k < kLanes; ++k) S->lane_worker[k] = std::thread(lane_loop, S, k);
    *out = S;
    return KOMA_OK;
}

extern "C" koma_status koma_server_submit(koma_server* S, int64_t n, const double* x, const double* y,
                                          const double* z, const double* pd, const double* t1, const double* t2,
                                          const double* dw, const int64_t* group_offsets, int64_t n_groups,
                                          int64_t n_steps, const double* dt, const double* gx, const double* gy,
                                          const double* gz, const double* b1_re, const double* b1_im,
                                          const uint8_t* adc, uint64_t* id_out) {
    NvtxRange nvtx_("koma_server_submit");
    if (!S || !id_out) return KOMA_E_INVALID;
    const koma::SerialHostScope serial_;  // submitters run side by side: no worker pool
    Req* r = new (std::nothrow) Req();
    if (!r) return KOMA_E_NOMEM;
    r->t_submit = now_s();
    std::string err;
    // the second lane (grouped requests, large ones): the spins are checked
    // and converted on the device below (or on the host when the phantom
    // cannot be placed on the device yet)
    const bool lane = (group_offsets && n_groups > 1) || (S->plain_spins > 0 && n >= S->plain_spins);
    int st = KOMA_OK;
    if (lane) {
        if (n < 0 || (n > 0 && (!x || !y || !z || !pd || !t1 || !t2 || !dw))) {
            st = KOMA_E_INVALID;
            err = "phantom: n < 0 or a NULL array";
        }
        r->n_pad = std::max<int64_t>(32, (n + 31) / 32 * 32);
    } else {
        st = koma::host_phantom32(n, x, y, z, pd, t1, t2, dw, r->h32, r->n_pad, r->max_abs, err);
    }
    if (st == KOMA_OK && group_offsets) {
        // the upload's rules: n_groups >= 1, offsets from 0 to n, non-decreasing
        bool ok = n_groups >= 1 && group_offsets[0] == 0 && group_offsets[n_groups] == n;
        for (int64_t g = 0; ok && g < n_groups; ++g) ok = group_offsets[g] <= group_offsets[g + 1];
        if (!ok) {
            st = KOMA_E_INVALID;
            err = "server_submit: group_offsets must run from 0 to n without decreasing (n_groups >= 1)";
        }
    }
    koma_sequence_info info{};
    if (st == KOMA_OK && lane) {
        st = koma::host_check_sequence(n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, info, err);
        // memory estimate without the records: at most one record per step
        // and time point, one readout snapshot row per block between RF runs
        info.n_records = n_steps + 1;
        info.n_adc_runs = std::min<int64_t>(info.n_adc, info.n_materialize + 1);
    } else if (st == KOMA_OK) {
        st = koma::host_records32(n_steps, dt, gx, gy, gz, b1_re, b1_im, adc, r->recs, info, err);
    }
    if (st != KOMA_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->fatal = err;
        delete r;
        return static_cast<koma_status>(st);
    }
    r->n = n;
    r->n_steps = n_steps;
    r->n_adc = info.n_adc;
    r->n_rec = info.n_records;
    r->n_adc_runs = info.n_adc_runs;
    r->n_groups = group_offsets ? n_groups : 1;
    r->lane = lane;
    if (r->lane) {
        // the phantom on the device now (checked and converted there), else
        // a host copy that the lane uploads
        if (n > 0) st = upload_lane_phantom(S, r, n, x, y, z, pd, t1, t2, dw, err);
        if (st == KOMA_E_NOMEM) {
            st = koma::host_check_phantom(n, x, y, z, pd, t1, t2, dw, err);
            const double* ph[7] = {x, y, z, pd, t1, t2, dw};
            if (st == KOMA_OK) {
                // not value-initialised: the copy is the only write
                r->ph64.reset(new (std::nothrow) double[static_cast<size_t>(7 * n)]);
                if (!r->ph64) st = KOMA_E_NOMEM;
            }
            for (int k = 0; k < 7 && st == KOMA_OK; ++k)
                std::memcpy(r->ph64.get() + k * n, ph[k], static_cast<size_t>(n) * sizeof(double));
        }
        if (st != KOMA_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->fatal = err;
            delete r;
            return static_cast<koma_status>(st);
        }
        if (group_offsets) {
            r->offsets.assign(group_offsets, group_offsets + n_groups + 1);
            // every group has one T1 and one T2 (a dictionary): relaxation once per thread
            bool uni = true;
            for (int64_t gi = 0; gi < n_groups && uni; ++gi)
                for (int64_t j = group_offsets[gi] + 1; j < group_offsets[gi + 1] && uni; ++j)
                    uni = t1[j] == t1[group_offsets[gi]] && t2[j] == t2[group_offsets[gi]];
            r->uni_relax = uni;
        }
        const int64_t v = n_steps + 1;
        r->sq64.resize(static_cast<size_t>(n_steps + 3 * v + 2 * n_steps));
        double* q = r->sq64.data();
        if (n_steps > 0) std::memcpy(q, dt, static_cast<size_t>(n_steps) * sizeof(double));
        std::memcpy(q + n_steps, gx, static_cast<size_t>(v) * sizeof(double));
        std::memcpy(q + n_steps + v, gy, static_cast<size_t>(v) * sizeof(double));
        std::memcpy(q + n_steps + 2 * v, gz, static_cast<size_t>(v) * sizeof(double));
        if (n_steps > 0) {
            std::memcpy(q + n_steps + 3 * v, b1_re, static_cast<size_t>(n_steps) * sizeof(double));
            std::memcpy(q + 2 * n_steps + 3 * v, b1_im, static_cast<size_t>(n_steps) * sizeof(double));
        }
        r->sq_adc.assign(adc, adc + v);
        r->recs.clear();
        r->recs.shrink_to_fit();
        r->units_total = 0;
        r->rem_work = 0;
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            if (r->dp64) cudaFreeAsync(r->dp64, S->s_red);
            if (r->dp32) cudaFreeAsync(r->dp32, S->s_red);
            S->used -= std::min(S->used, r->ph_dev_bytes);
            delete r;
            return KOMA_E_BUSY;
        }
        r->prep_s = now_s() - r->t_submit;
        r->id = S->next_id++;
        S->all[r->id] = r;
        S->pending.push_back(r);
        S->submitted++;
        *id_out = r->id;
        S->cv_work.notify_all();
        return KOMA_OK;
    }
    for (int d = 0; d < 4; ++d) {
        r->ext[d] = static_cast<float>(r->max_abs[d] * (1.0 + 1e-6));
        if (r->max_abs[d] > 0) r->used |= 1 << d;
    }
    r->n_batches = (r->n_adc > 0 && n > 0) ? (n + kBatchSpins - 1) / kBatchSpins : 0;
    koma::host_rf_maps32(r->recs, r->pulses, info);
    if (!r->pulses.empty()) {
        // the batches walk the compacted stream (a repeated pulse is one
        // REC_MAP record); the map kernel steps the pulses from the full one
        r->recs_full.swap(r->recs);
        koma::compact_records32(r->recs_full, r->recs);
        r->n_rec = static_cast<int64_t>(r->recs.size());
    }
    r->chunk = S->chunk;
    r->chunk_begin.clear();
    for (int64_t b = 0; b < r->n_rec; b += r->chunk) r->chunk_begin.push_back(b);
    if (r->chunk_begin.empty()) r->chunk_begin.push_back(0);
    r->chunk_begin.push_back(r->n_rec);
    r->n_chunks = static_cast<int64_t>(r->chunk_begin.size()) - 1;
    r->chunk_work.assign(static_cast<size_t>(r->n_chunks), 0.0);
    r->chunk_hdr.assign(static_cast<size_t>(r->n_chunks), -1);
    int64_t hdr = -1;
    for (int64_t c = 0; c < r->n_chunks; ++c) {
        for (int64_t i = r->chunk_begin[c]; i < r->chunk_begin[c + 1]; ++i) {
            const koma::Rec32& q = r->recs[static_cast<size_t>(i)];
            if (i == r->chunk_begin[c] && q.type == koma::REC_RF && q.count == 0) r->chunk_hdr[c] = hdr;
            if (q.type == koma::REC_RF && q.count > 0) hdr = i;
            r->chunk_work[c] += q.type == koma::REC_ADC ? 1.0 + (q.count & koma::kCountMask) / 8.0 : 1.0;
        }
    }
    double w = 0;
    for (double cw : r->chunk_work) w += cw;
    r->work_per_spin = std::max(1.0, w);
    r->units_total = r->n_batches * r->n_chunks;
    r->batch_next.assign(static_cast<size_t>(r->n_batches), 0);
    r->batch_busy.assign(static_cast<size_t>(r->n_batches), 0);
    r->rem_work = static_cast<double>(r->n_batches) * kBatchSpins * w;
    upload_shared_request(S, r);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
        if (r->uploaded) {
            cudaEventSynchronize(r->ev_up);  // its copies are done
            release_device(S, r);
            host_release(S, r);
            cudaEventDestroy(r->ev_up);
            cudaEventDestroy(r->ev_done);
        }
        delete r;
        return KOMA_E_BUSY;
    }
    r->prep_s = now_s() - r->t_submit;
    r->id = S->next_id++;
    S->all[r->id] = r;
    S->pending.push_back(r);
    S->submitted++;
    *id_out = r->id;
    S->cv_work.notify_all();
    return KOMA_OK;
}

extern "C" koma_status koma_server_wait(koma_server* S, uint64_t id, double timeout_s, double* sig_host,
                                        int64_t capacity, koma_request_info* info) {
    if (!S) return KOMA_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return KOMA_E_INVALID;
    Req* r = it->second;
    auto finished = [&] { return (r->state == DONE || r->state == FAILED) && r->t_done >= 0 && r->retired; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, finished);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
        return KOMA_E_TIMEOUT;
    }
    if (info) {
        info->id = r->id;
        info->n_groups = r->n_groups;
        info->lane = r->lane ? 1 : 0;
        info->prep_s = r->prep_s;
        info->upload_s = r->upload_s;
        info->run_s = r->run_s;
        info->n_spins = r->n;
        info->n_steps = r->n_steps;
        info->n_adc = r->n_adc;
        info->submit_s = r->t_submit - S->t0;
        info->admit_s = r->t_admit >= 0 ? r->t_admit - S->t0 : -1;
        info->done_s = r->t_done - S->t0;
        info->latency_s = r->t_done - r->t_submit;
        info->launches = r->launches;
        info->status = r->state == DONE ? KOMA_OK : r->err;
    }
    koma_status st = r->state == DONE ? KOMA_OK : r->err;
    if (st == KOMA_OK && r->n_adc > 0) {
        const int64_t total = r->n_groups * r->n_adc;
        if (!sig_host || capacity < total) return KOMA_E_INVALID;  // keep the result for a retry
        std::memcpy(sig_host, r->hsig, static_cast<size_t>(total) * 2 * sizeof(double));
    } else if (st == KOMA_OK && sig_host && capacity > 0) {
        // nothing observed
    }
    if (st != KOMA_OK) S->fatal = r->msg;
    S->all.erase(it);
    lk.unlock();
    host_release(S, r);  // the result's copy into it completed before the request was retired
    if (r->ev_up) cudaEventDestroy(r->ev_up);
    if (r->ev_done) cudaEventDestroy(r->ev_done);
    delete r;
    return st;
}

extern "C" koma_status koma_server_get_stats(koma_server* S, koma_server_stats* out) {
    if (!S || !out) return KOMA_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->pending = static_cast<int64_t>(S->pending.size());
    out->active = static_cast<int64_t>(S->active.size());
    out->launches = S->launches;
    out->batches = S->batches;
    out->mem_used = S->used;
    out->mem_peak = S->peak;
    out->lane_runs = S->lane_runs;
    return KOMA_OK;
}

extern "C" const char* koma_server_last_error(const koma_server* S) { return S ? S->fatal.c_str() : "null server"; }

extern "C" koma_status koma_server_destroy(koma_server* S) {
    if (!S) return KOMA_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Req* r : S->pending) fail_req(r, KOMA_E_BUSY, "server shut down before admission");
        for (Req* r : S->pending) {
            r->t_done = now_s();
            r->retired = true;
            S->failed++;
        }
        S->pending.clear();
        S->cv_work.notify_all();
        S->cv_done.notify_all();
        S->cv_lane.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (int k = 0; k < kLanes; ++k) {
        if (S->lane_worker[k].joinable()) S->lane_worker[k].join();
        if (S->lane_ctx[k]) koma_destroy(S->lane_ctx[k]);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    if (S->s_red) cudaStreamSynchronize(S->s_red);
    for (Slot& sl : S->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_buf) cudaFreeHost(sl.h_buf);
        if (sl.d_buf) cudaFree(sl.d_buf);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    for (auto& kv : S->all) {
        Req* r = kv.second;
        if (r->hsig) cudaFreeHost(r->hsig);
        if (r->ev_up) cudaEventDestroy(r->ev_up);
        if (r->ev_done) cudaEventDestroy(r->ev_done);
        delete r;
    }
    for (auto& v : S->host_free)
        for (void* p : v) cudaFreeHost(p);
    for (koma_server::UpSlot* U : S->up_all) {
        cudaStreamSynchronize(U->st);
        cudaStreamDestroy(U->st);
        cudaFree(U->d_cs);
        cudaFreeHost(U->h_cs);
        delete U;
    }
    S->up_all.clear();
    S->up_free.clear();
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->s_up) cudaStreamDestroy(S->s_up);
    if (S->s_red) cudaStreamDestroy(S->s_red);
    for (int k = 0; k < kLanes; ++k)
        if (S->s_lane[k]) cudaStreamDestroy(S->s_lane[k]);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
    return KOMA_OK;
}
