// server.cu -- continuous-batching permanent server (host side).
//
// Requests of any order and element type arrive through perm_submit and are
// completed asynchronously.  A worker thread drives three lanes on their own
// CUDA streams, so their work overlaps on the device:
//
//   fast lane   complex orders n <= 20 (Store-zechin, one CTA per matrix or
//               the layer path) and integer orders n <= 28 (Ryser): every
//               pending request of this kind joins the next batch as soon as
//               the lane's previous batch has finished (continuous batching).
//               Highest stream priority.
//   table lane  complex orders 21..34 whose Store-zechin chain tables (the
//               "stored sub-permanents" of Section 4 of Su & Zheng,
//               arXiv:1802.02779) fit the table budget.  Up to kTableSlots
//               jobs run at once, each on its own stream; a job is the request
//               at the head of the queue plus the queued requests of the same
//               order behind it (they share every layer launch).  A job is
//               admitted while the tables of all jobs in flight stay within
//               the budget -- C(t, t/2) chains of 2^12 or 2^13 entries, two
//               layers, per matrix.  Its tables are a contiguous range of
//               one allocation of the budget's size, made when the server is
//               created and carved on the host (first fit), and the range
//               returns when the job's kernels are seen to finish, so the next
//               job is admitted as memory frees up -- no allocation call on the
//               worker's path.  Middle priority.
//   Ryser lane  every other order (Ryser's formula, Section 3.3, which needs no
//               tables): batches of pending requests, grouped by order inside
//               one perm_batch, bounded by their number of Gray codes.  Lowest
//               priority.
//
// The large lanes launch one CTA per chain or per piece of Gray codes, so
// their CTAs retire every few milliseconds and a batch that arrives on a
// higher-priority lane takes the freed SM slots first.  The worker never
// blocks on the device: it polls events, so a stuck lane cannot hang the
// host; perm_server_destroy waits at most timeout_ms.
#include "perm_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace perm;

perm_status plan_create_impl(int n_max, perm_dtype dtype, const perm_opts* opts, void* ext_ws,
                             size_t ext_ws_bytes, perm_plan_t* out);

namespace {

constexpr int kFastComplexN = 20;        // complex orders of the fast lane
constexpr int kFastIntN = 28;            // integer orders of the fast lane (Ryser, <= 1 ms each)
constexpr int kQueueCap = 1 << 16;
constexpr int kFastBatch = 4096;
constexpr int kTableSlots = 4;           // table-lane jobs in flight at once
constexpr int kTableJob = 16;            // requests of one order per table job
constexpr int kRyserBatch = 64;
// A Ryser batch holds requests up to 2^31 complex-code equivalents of work (about 0.7 s; a
// larger request runs alone): every request of a batch completes with the batch, so a large
// request must not hold small ones back.  An integer code costs about a tenth of a complex one.
constexpr double kRyserBatchCodes = 2147483648.0;
constexpr size_t kResultSlot = 32;       // bytes reserved per result in the slot buffers

enum { kLaneFast = 0, kLaneTable = 1, kLaneRyser = 2, kLanes = 3 };

struct Request {
    uint64_t ticket = 0;
    int n = 0;
    int dtype = PERM_C128;
    std::vector<unsigned char> mat;       // host copy of the input
    std::atomic<int> state{0};            // 0 queued, 1 on device, 2 done
    unsigned char result[32] = {0};
    int result_bytes = 16;                // 32 for integers on a PERM_FLAG_WIDE server
    int status = PERM_OK;
};

size_t elem_bytes(int dtype) { return dtype == PERM_C128 ? 16 : 8; }
int dtype_slot(int dtype) { return dtype == PERM_C128 ? 0 : (dtype == PERM_U01 ? 1 : 2); }

// One unit of work in flight: its stream, completion event and buffers.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char* h_in = nullptr;   // pinned staging of the inputs
    unsigned char* d_in = nullptr;
    size_t in_cap = 0;
    unsigned char* h_out = nullptr;  // pinned results (up to 32 B each) and statuses
    unsigned char* d_out = nullptr;
    int* h_status = nullptr;
    int* d_status = nullptr;
    int out_cap = 0;
    ItemDesc* h_desc = nullptr;      // table slots: descriptors of the job's matrices
    ItemDesc* d_desc = nullptr;
    unsigned* d_counter = nullptr;   // table slots: work counter of a dataflow launch
    size_t ws_off = 0;               // table slots: the job's tables in the arena
    size_t ws_bytes = 0;
    std::vector<Request*> inflight;
    std::vector<size_t> inflight_at;  // byte offset of each in-flight result in h_out
    bool busy = false;
};

struct Lane {
    int priority = 0;
    int method = PERM_METHOD_AUTO;
    int max_batch = 1;
    perm_plan_t plans[3] = {nullptr, nullptr, nullptr};   // by dtype slot (fast and Ryser lanes)
    int n_max[3] = {0, 0, 0};
    std::vector<Slot> slots;
};

}  // namespace

struct perm_server_s {
    perm_opts opts{};
    int device = 0;
    int num_sms = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queues[kLanes];
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    int queued = 0;
    std::atomic<bool> stop{false};
    std::atomic<bool> failed{false};
    std::atomic<bool> abandon{false};   // process exit: the worker stops touching the device
    std::atomic<int> busy_slots{0};
    std::thread worker;
    Lane lanes[kLanes];
    size_t table_budget = 0;
    unsigned char* arena = nullptr;     // the table lane's memory (table_budget bytes)
    std::map<size_t, size_t> arena_free; // free ranges of the arena: offset -> bytes (worker only)
    int queue_cap = kQueueCap;
};

namespace {

// Servers whose perm_server_destroy timed out keep draining on their worker
// thread.  At process exit those workers are told to stop and are joined before
// the CUDA runtime tears itself down: the handler is registered with atexit
// after the runtime was initialised, so it runs before the runtime's own exit
// handlers.  The worker never waits on the device, so the join is prompt.
std::mutex g_leaked_mu;
std::vector<perm_server_t> g_leaked;
std::once_flag g_leaked_once;

void stop_leaked_workers() {
    std::vector<perm_server_t> v;
    {
        std::lock_guard<std::mutex> g(g_leaked_mu);
        v.swap(g_leaked);
    }
    for (perm_server_t s : v) {
        s->abandon.store(true);
        s->cv.notify_all();
        if (s->worker.joinable()) s->worker.join();
    }
}

bool slot_alloc(Slot& S, int priority, size_t in_cap, int out_cap, int descs) {
    if (cudaStreamCreateWithPriority(&S.stream, cudaStreamNonBlocking, priority) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess) return false;
    S.in_cap = in_cap;
    S.out_cap = out_cap;
    if (cudaMallocHost(&S.h_in, in_cap) != cudaSuccess) return false;
    if (cudaMalloc(&S.d_in, in_cap) != cudaSuccess) return false;
    if (cudaMallocHost(&S.h_out, (size_t)out_cap * kResultSlot) != cudaSuccess) return false;
    if (cudaMalloc(&S.d_out, (size_t)out_cap * kResultSlot) != cudaSuccess) return false;
    if (cudaMallocHost(&S.h_status, (size_t)out_cap * sizeof(int)) != cudaSuccess) return false;
    if (cudaMalloc(&S.d_status, (size_t)out_cap * sizeof(int)) != cudaSuccess) return false;
    if (descs > 0) {
        if (cudaMallocHost(&S.h_desc, (size_t)descs * sizeof(ItemDesc)) != cudaSuccess) return false;
        if (cudaMalloc(&S.d_desc, (size_t)descs * sizeof(ItemDesc)) != cudaSuccess) return false;
        if (cudaMalloc(&S.d_counter, 64) != cudaSuccess) return false;
    }
    return true;
}

void slot_free(Slot& S) {
    if (S.d_in) cudaFree(S.d_in);
    if (S.d_out) cudaFree(S.d_out);
    if (S.d_status) cudaFree(S.d_status);
    if (S.d_desc) cudaFree(S.d_desc);
    if (S.d_counter) cudaFree(S.d_counter);
    if (S.h_in) cudaFreeHost(S.h_in);
    if (S.h_out) cudaFreeHost(S.h_out);
    if (S.h_status) cudaFreeHost(S.h_status);
    if (S.h_desc) cudaFreeHost(S.h_desc);
    if (S.done) cudaEventDestroy(S.done);
    if (S.stream) cudaStreamDestroy(S.stream);
    S = Slot();
}

void lane_free(Lane& L) {
    for (auto& p : L.plans)
        if (p) { perm_plan_destroy(p); p = nullptr; }
    for (auto& S : L.slots) slot_free(S);
    L.slots.clear();
}

perm_plan_t lane_plan(perm_server_t s, Lane& L, int dtype) {
    const int k = dtype_slot(dtype);
    if (!L.plans[k]) {
        perm_opts o{};
        o.flags = dtype == PERM_C128 ? 0u : (s->opts.flags & PERM_FLAG_WIDE);
        o.method = L.method;
        o.max_batch = L.max_batch;
        perm_plan_t p = nullptr;
        if (plan_create_impl(L.n_max[k], (perm_dtype)dtype, &o, nullptr, 0, &p) != PERM_OK) return nullptr;
        L.plans[k] = p;
    }
    return L.plans[k];
}

// Table bytes of a job of `count` complex matrices of order n on the table lane (the layer
// path's default shape for that order and count).
int table_low(int n, int count) {
    int m = 0, threads = 0;
    sz_layer_default_shape(n, count, &m, &threads);
    return m;
}
// Jobs of at most kFlowMaxCount matrices of an order up to kLayerSmallN run as one dataflow launch.
bool table_flow(int n, int count) { return n <= kLayerSmallN && count <= kFlowMaxCount; }
size_t table_item_bytes(int n, int count) {
    const int m = table_low(n, count);
    return table_flow(n, count) ? sz_flow_workspace_bytes(n, m) : sz_matrix_workspace_bytes(PERM_C128, n, m);
}
size_t table_bytes(int n, int count) { return (size_t)count * table_item_bytes(n, count); }
// The most one matrix of order n can take (admission to the table lane).
size_t table_bytes_max(int n) {
    size_t b = 0;
    for (int c = 1; c <= kFlowMaxCount + 1; c++) b = std::max(b, table_item_bytes(n, c));
    return b;
}

// Work of one request on the Ryser lane in complex-code equivalents (the batch bound).
double ryser_codes(const Request* r) {
    const double codes = std::ldexp(1.0, r->dtype == PERM_I64 ? r->n : std::max(0, r->n - 1));
    return r->dtype == PERM_C128 ? codes : 0.1 * codes;
}

// Copy results back and record the slot's completion event.
bool slot_finish_launch(Slot& S, size_t out_bytes, int nout) {
    if (cudaMemcpyAsync(S.h_out, S.d_out, out_bytes, cudaMemcpyDeviceToHost, S.stream) != cudaSuccess)
        return false;
    if (cudaMemcpyAsync(S.h_status, S.d_status, (size_t)nout * sizeof(int), cudaMemcpyDeviceToHost,
                        S.stream) != cudaSuccess)
        return false;
    return cudaEventRecord(S.done, S.stream) == cudaSuccess;
}

// Fast and Ryser lanes: the requests `batch` through the lane's plans, one
// perm_batch per dtype, inputs packed per dtype group; each group's results are
// packed at its own slot size (16 B, or 32 B for wide integers).
bool plan_launch(perm_server_t s, Lane& L, Slot& S, std::vector<Request*>& batch) {
    size_t off = 0, out_off = 0;
    int outpos = 0;
    S.inflight.clear();
    S.inflight_at.clear();
    for (int slot = 0; slot < 3; slot++) {
        const int dtype = slot == 0 ? PERM_C128 : (slot == 1 ? PERM_U01 : PERM_I64);
        const size_t rbytes = (dtype != PERM_C128 && (s->opts.flags & PERM_FLAG_WIDE)) ? 32 : 16;
        std::vector<int> sizes;
        const size_t start = off;
        const size_t out_start = out_off;
        const int status_start = outpos;
        for (Request* r : batch) {
            if (r->dtype != dtype) continue;
            std::memcpy(S.h_in + off, r->mat.data(), r->mat.size());
            off += r->mat.size();
            sizes.push_back(r->n);
            r->result_bytes = (int)rbytes;
            S.inflight.push_back(r);
            S.inflight_at.push_back(out_off);
            out_off += rbytes;
            outpos++;
        }
        if (sizes.empty()) continue;
        perm_plan_t p = lane_plan(s, L, dtype);
        if (!p) return false;
        if (off > start && cudaMemcpyAsync(S.d_in + start, S.h_in + start, off - start,
                                           cudaMemcpyHostToDevice, S.stream) != cudaSuccess)
            return false;
        if (perm_batch(p, S.d_in + start, sizes.data(), (int)sizes.size(), S.d_out + out_start,
                       S.d_status + status_start, S.stream) != PERM_OK)
            return false;
    }
    if (!slot_finish_launch(S, out_off, outpos)) return false;
    for (Request* r : batch) r->state.store(1, std::memory_order_relaxed);
    S.busy = true;
    return true;
}

// The table lane's arena (worker thread only): first-fit ranges of the one
// allocation, sizes rounded to 256 bytes, neighbours merged when freed.
constexpr size_t kArenaAlign = 256;
size_t arena_round(size_t bytes) { return (bytes + kArenaAlign - 1) & ~(kArenaAlign - 1); }

size_t arena_largest(const perm_server_t s) {
    size_t best = 0;
    for (const auto& f : s->arena_free) best = std::max(best, f.second);
    return best;
}

bool arena_alloc(perm_server_t s, size_t bytes, size_t* off) {
    bytes = arena_round(bytes);
    for (auto it = s->arena_free.begin(); it != s->arena_free.end(); ++it) {
        if (it->second < bytes) continue;
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        s->arena_free.erase(it);
        if (rest) s->arena_free.emplace(at, rest);
        return true;
    }
    return false;
}

void arena_release(perm_server_t s, size_t off, size_t bytes) {
    bytes = arena_round(bytes);
    auto it = s->arena_free.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != s->arena_free.end() && it->first + it->second == next->first) {
        it->second += next->second;
        s->arena_free.erase(next);
    }
    if (it != s->arena_free.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            s->arena_free.erase(it);
        }
    }
}

// Table lane: one job (requests of one order) on the slot's stream, its tables
// a range of the arena that take_table_job found free.  Returns false on a CUDA
// error (the range is then returned).
bool table_launch(perm_server_t s, Slot& S, std::vector<Request*>& job) {
    const int n = job[0]->n;
    const int c = (int)job.size();
    const size_t ws_item = table_item_bytes(n, c);
    S.inflight.clear();
    S.inflight_at.clear();
    size_t off = 0;
    for (int i = 0; i < c; i++) {
        Request* r = job[i];
        std::memcpy(S.h_in + off, r->mat.data(), r->mat.size());
        S.h_desc[i] = ItemDesc{(long long)(off / 16), n, i};
        off += r->mat.size();
        r->result_bytes = 16;
        S.inflight.push_back(r);
        S.inflight_at.push_back((size_t)i * 16);
    }
    size_t ws_off = 0;
    if (!arena_alloc(s, (size_t)c * ws_item, &ws_off)) return false;   // take_table_job checked the fit
    void* ws = s->arena + ws_off;
    bool ok = cudaMemcpyAsync(S.d_in, S.h_in, off, cudaMemcpyHostToDevice, S.stream) == cudaSuccess &&
              cudaMemcpyAsync(S.d_desc, S.h_desc, (size_t)c * sizeof(ItemDesc), cudaMemcpyHostToDevice,
                              S.stream) == cudaSuccess;
    int lm = 0, lthreads = 0;
    sz_layer_default_shape(n, c, &lm, &lthreads);
    // small jobs: one dataflow launch (a few milliseconds at most); others: one CTA per chain (no
    // CTA loops over several), so CTAs retire every chain and a batch of the fast lane waits at
    // most a chain's time for SMs, not a whole layer launch's
    if (ok && table_flow(n, c))
        ok = sz_launch_flow(S.d_in, S.d_desc, c, n, lm, S.d_out, S.d_status, ws, ws_item, S.d_counter,
                            s->num_sms, S.stream) == cudaSuccess;
    else if (ok)
        ok = sz_launch_layers(PERM_C128, S.d_in, S.d_desc, c, n, lm, S.d_out, 2, S.d_status, ws, ws_item,
                              1 << 30, S.stream, lthreads) == cudaSuccess;
    if (ok) ok = slot_finish_launch(S, (size_t)c * 16, c);
    if (!ok) {
        arena_release(s, ws_off, (size_t)c * ws_item);
        return false;
    }
    for (Request* r : job) r->state.store(1, std::memory_order_relaxed);
    S.ws_off = ws_off;
    S.ws_bytes = (size_t)c * ws_item;
    S.busy = true;
    return true;
}

void slot_complete(Slot& S) {
    for (size_t i = 0; i < S.inflight.size(); i++) {
        Request* r = S.inflight[i];
        std::memcpy(r->result, S.h_out + S.inflight_at[i], (size_t)r->result_bytes);
        r->status = S.h_status[i];
        r->state.store(2, std::memory_order_release);
    }
    S.inflight.clear();
    S.inflight_at.clear();
    S.busy = false;
}

void fail_requests(std::vector<Request*>& v) {
    for (Request* r : v) { r->status = PERM_ECUDA; r->state.store(2, std::memory_order_release); }
}

// Take requests for the fast or the Ryser lane (caller holds s->mu).
void take_batch(perm_server_t s, int li, const Slot& S, std::vector<Request*>& batch) {
    auto& q = s->queues[li];
    size_t bytes = 0;
    double codes = 0.0;
    const size_t cap = li == kLaneFast ? (size_t)kFastBatch : (size_t)kRyserBatch;
    while (!q.empty() && batch.size() < cap && batch.size() < (size_t)S.out_cap) {
        Request* r = q.front();
        if (bytes + r->mat.size() > S.in_cap) break;
        if (li == kLaneRyser && !batch.empty() && codes + ryser_codes(r) > kRyserBatchCodes) break;
        bytes += r->mat.size();
        codes += ryser_codes(r);
        batch.push_back(r);
        q.pop_front();
    }
    s->queued -= (int)batch.size();
}

// Take one table job (caller holds s->mu): the head of the queue, if its tables
// fit what the jobs in flight leave of the budget (first come, first served:
// nothing overtakes a head that does not fit yet), plus queued requests of the
// same order while their tables fit too.
void take_table_job(perm_server_t s, std::vector<Request*>& job) {
    auto& q = s->queues[kLaneTable];
    if (q.empty()) return;
    const int n = q.front()->n;
    const size_t avail = arena_largest(s);      // the job's tables are one contiguous range
    for (auto it = q.begin(); it != q.end() && (int)job.size() < kTableJob;) {
        Request* r = *it;
        if (r->n != n) { ++it; continue; }
        const int c = (int)job.size() + 1;
        if (arena_round(table_bytes(n, c)) > avail) break;
        job.push_back(r);
        it = q.erase(it);
    }
    s->queued -= (int)job.size();
}

void worker_loop(perm_server_t s) {
    cudaSetDevice(s->device);
    std::vector<Request*> batch;
    while (true) {
        if (s->abandon.load()) break;
        bool did = false;
        // completions
        for (int li = 0; li < kLanes; li++) {
            for (Slot& S : s->lanes[li].slots) {
                if (!S.busy) continue;
                const cudaError_t q = cudaEventQuery(S.done);
                if (q == cudaSuccess) {
                    slot_complete(S);
                    if (li == kLaneTable) {   // the job's kernels are done: its tables are free
                        arena_release(s, S.ws_off, S.ws_bytes);
                        S.ws_bytes = 0;
                    }
                    s->busy_slots--;
                    did = true;
                } else if (q != cudaErrorNotReady) {
                    s->failed = true;
                }
            }
        }
        if (s->failed.load()) {
            // a device error: fail everything that is still queued
            std::lock_guard<std::mutex> g(s->mu);
            for (auto& q : s->queues) {
                for (Request* r : q) { r->status = PERM_ECUDA; r->state.store(2, std::memory_order_release); }
                q.clear();
            }
            s->queued = 0;
        }
        // new work, highest priority first
        for (int li = 0; li < kLanes && !s->failed.load(); li++) {
            Lane& L = s->lanes[li];
            for (Slot& S : L.slots) {
                if (S.busy || s->failed.load()) continue;
                batch.clear();
                {
                    std::lock_guard<std::mutex> g(s->mu);
                    if (li == kLaneTable) take_table_job(s, batch);
                    else take_batch(s, li, S, batch);
                }
                if (batch.empty()) break;      // nothing (more) this lane can start now
                did = true;
                if (li == kLaneTable) {
                    if (table_launch(s, S, batch)) {
                        s->busy_slots++;
                    } else {
                        s->failed = true;
                        fail_requests(batch);
                    }
                } else if (plan_launch(s, L, S, batch)) {
                    s->busy_slots++;
                } else {
                    s->failed = true;
                    fail_requests(batch);
                }
            }
        }
        const bool idle = s->busy_slots.load() == 0;
        if (s->stop.load() && idle) {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->queued == 0) break;
        }
        if (s->stop.load() && s->failed.load()) break;
        if (!did) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(idle ? 500 : 20));
        }
    }
}

}  // namespace

extern "C" {

perm_status perm_server_create(const perm_opts* opts, void* stream, perm_server_t* out) {
    (void)stream;   // the server owns its streams
    if (!out) return PERM_EINVAL;
    *out = nullptr;
    perm_server_t s = new (std::nothrow) perm_server_s();
    if (!s) return PERM_ENOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.max_batch > 0) s->queue_cap = s->opts.max_batch;
    size_t free_b = 0, total_b = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete s;
        return PERM_ECUDA;
    }
    // table budget of the table lane: default min(100 GB, 40 % of the free memory), which holds
    // the compact tables of one n = 34 matrix (92.5 GB) on an otherwise idle GB300
    s->table_budget = s->opts.mem_budget_bytes ? s->opts.mem_budget_bytes
                                               : std::min<size_t>((size_t)100 << 30, (size_t)(0.4 * (double)free_b));
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    Lane& fast = s->lanes[kLaneFast];
    Lane& table = s->lanes[kLaneTable];
    Lane& ryser = s->lanes[kLaneRyser];
    fast.priority = greatest;
    fast.max_batch = kFastBatch;
    fast.n_max[0] = kFastComplexN;
    fast.n_max[1] = fast.n_max[2] = kFastIntN;
    table.priority = (least + greatest) / 2;
    ryser.priority = least;
    ryser.method = PERM_METHOD_RYSER;
    ryser.max_batch = kRyserBatch;
    ryser.n_max[0] = ryser.n_max[1] = ryser.n_max[2] = kMaxN;
    fast.slots.resize(1);
    table.slots.resize(kTableSlots);
    ryser.slots.resize(1);
    const size_t fast_in = (size_t)kFastBatch * std::max<size_t>(kFastComplexN * kFastComplexN * 16,
                                                                 kFastIntN * kFastIntN * 8);
    bool ok = slot_alloc(fast.slots[0], fast.priority, fast_in, kFastBatch, 0) &&
              slot_alloc(ryser.slots[0], ryser.priority, (size_t)kRyserBatch * kMaxN * kMaxN * 16, kRyserBatch, 0);
    for (Slot& S : table.slots)
        if (ok) ok = slot_alloc(S, table.priority, (size_t)kTableJob * kMaxNSZ * kMaxNSZ * 16, kTableJob, kTableJob);
    // the table lane's arena: all of the budget, allocated once
    if (ok) ok = cudaMalloc(&s->arena, s->table_budget) == cudaSuccess;
    if (ok) s->arena_free.emplace(0, s->table_budget & ~(kArenaAlign - 1));
    // the plans now (they load their kernels): creating one, or loading a kernel, while another
    // lane's work runs could wait for that work; the table lane's kernels are loaded here too
    for (int dt : {PERM_C128, PERM_U01, PERM_I64}) {
        if (ok) ok = lane_plan(s, fast, dt) != nullptr;
        if (ok) ok = lane_plan(s, ryser, dt) != nullptr;
    }
    if (ok) ok = sz_init_tables() == cudaSuccess && sz_preload(PERM_C128) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (auto& L : s->lanes) lane_free(L);
        if (s->arena) cudaFree(s->arena);
        delete s;
        return PERM_ENOMEM;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return PERM_OK;
}

perm_status perm_submit(perm_server_t s, const void* host_mat, int n, perm_dtype dtype, uint64_t* ticket) {
    if (!s || !ticket || n < 0 || n > kMaxN || (n > 0 && !host_mat)) return PERM_EINVAL;
    if (dtype != PERM_C128 && dtype != PERM_U01 && dtype != PERM_I64) return PERM_EINVAL;
    if (s->stop.load()) return PERM_ESHUTDOWN;
    if (s->failed.load()) return PERM_ECUDA;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return PERM_ENOMEM;
    r->n = n;
    r->dtype = dtype;
    const size_t bytes = (size_t)n * n * elem_bytes(dtype);
    r->mat.resize(bytes);
    if (bytes) std::memcpy(r->mat.data(), host_mat, bytes);
    // lane by cost: small orders batch on the fast lane; complex orders whose Store-zechin
    // tables fit the budget on the table lane; everything else with Ryser
    int lane;
    if (n <= (dtype == PERM_C128 ? kFastComplexN : kFastIntN)) lane = kLaneFast;
    else if (auto_uses_sz(dtype) && n <= kMaxNSZ && table_bytes_max(n) + ((size_t)1 << 20) <= s->table_budget)
        lane = kLaneTable;
    else lane = kLaneRyser;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->queued >= s->queue_cap) return PERM_EAGAIN;
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        Request* raw = r.get();
        s->queues[lane].push_back(raw);
        s->queued++;
        s->reqs.emplace(raw->ticket, std::move(r));
    }
    s->cv.notify_one();
    return PERM_OK;
}

perm_status perm_poll(perm_server_t s, uint64_t ticket, void* out, int* item_status) {
    if (!s || !out) return PERM_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PERM_ENOTFOUND;
    Request* r = it->second.get();
    if (r->state.load(std::memory_order_acquire) != 2) return PERM_EAGAIN;
    std::memcpy(out, r->result, (size_t)r->result_bytes);
    if (item_status) *item_status = r->status;
    const int st = r->status == PERM_ECUDA ? PERM_ECUDA : PERM_OK;
    s->reqs.erase(it);
    return (perm_status)st;
}

perm_status perm_server_destroy(perm_server_t s, int timeout_ms) {
    if (!s) return PERM_OK;
    s->stop.store(true);
    s->cv.notify_all();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    perm_status result = PERM_OK;
    // wait for the worker to drain, bounded
    while (true) {
        bool busy;
        {
            std::lock_guard<std::mutex> g(s->mu);
            busy = s->busy_slots.load() > 0 || s->queued > 0;
        }
        if (!busy || s->failed.load()) break;
        if (std::chrono::steady_clock::now() >= deadline) { result = PERM_ETIMEDOUT; break; }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    if (result == PERM_ETIMEDOUT) {
        // leave the device work alone: the worker keeps draining in the background and
        // the server object is leaked rather than freed under running kernels
        std::call_once(g_leaked_once, [] { std::atexit(stop_leaked_workers); });
        std::lock_guard<std::mutex> g(g_leaked_mu);
        g_leaked.push_back(s);
        return PERM_ETIMEDOUT;
    }
    s->worker.join();
    for (auto& L : s->lanes) lane_free(L);
    if (s->arena) cudaFree(s->arena);
    delete s;
    return result;
}

}  // extern "C"
