// server.cu -- continuous-batching permanent server (host side).
//
// Requests of any order and element type arrive through perm_submit and are
// completed asynchronously.  A worker thread drives three lanes, each with its
// own CUDA stream, so their work overlaps on the device:
//
//   batch lane  orders n <= kSmallN: every pending request of this kind is
//               taken into the next batch as soon as the previous batch of the
//               lane has finished (continuous batching); complex matrices by
//               Store-zechin with one CTA per matrix, integers by Ryser.
//               Highest stream priority.
//   table lane  complex orders n > kSmallN whose Store-zechin chain tables
//               (the "stored sub-permanents" of Section 4 of Su & Zheng,
//               arXiv:1802.02779) fit the table budget: admitted one at a
//               time into the budget.  Middle priority.
//   Ryser lane  the other orders n > kSmallN (and every larger integer
//               order): Ryser's formula (Section 3.3), which needs no
//               tables.  Lowest priority.
//
// The large lanes launch one CTA per chain or per piece of Gray codes, so
// their CTAs retire every few milliseconds and a batch that arrives on the
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

constexpr int kSmallN = 20;
constexpr int kQueueCap = 1 << 16;
constexpr int kLaneBatch = 4096;
constexpr int kLargeLow = 13;      // chain width of the one-matrix Store-zechin path

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

struct Lane {
    cudaStream_t stream = nullptr;
    int priority = 0;
    int method = PERM_METHOD_AUTO;
    cudaEvent_t done = nullptr;
    perm_plan_t plans[3] = {nullptr, nullptr, nullptr};   // by dtype slot
    int n_max = 0;
    void* ext_ws = nullptr;          // large lane: shared Store-zechin workspace
    size_t ext_ws_bytes = 0;
    unsigned char* h_in = nullptr;   // pinned staging of one batch's inputs
    unsigned char* d_in = nullptr;
    size_t in_cap = 0;
    unsigned char* h_out = nullptr;  // pinned results (up to 32 B each) and statuses
    unsigned char* d_out = nullptr;
    int* h_status = nullptr;
    int* d_status = nullptr;
    int out_cap = 0;
    std::vector<Request*> inflight;
    std::vector<size_t> inflight_at;  // byte offset of each in-flight result in h_out
    std::atomic<bool> busy{false};
};

constexpr size_t kResultSlot = 32;   // bytes reserved per result in the lane buffers

}  // namespace

struct perm_server_s {
    perm_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queues[3];
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    int queued = 0;
    std::atomic<bool> stop{false};
    std::atomic<bool> failed{false};
    std::atomic<bool> abandon{false};   // process exit: the worker stops touching the device
    std::thread worker;
    Lane lanes[3];
    size_t table_budget = 0;
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

bool lane_alloc(Lane& L, size_t in_cap, int out_cap) {
    if (cudaStreamCreateWithPriority(&L.stream, cudaStreamNonBlocking, L.priority) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) return false;
    L.in_cap = in_cap;
    L.out_cap = out_cap;
    if (cudaMallocHost(&L.h_in, in_cap) != cudaSuccess) return false;
    if (cudaMalloc(&L.d_in, in_cap) != cudaSuccess) return false;
    if (cudaMallocHost(&L.h_out, (size_t)out_cap * kResultSlot) != cudaSuccess) return false;
    if (cudaMalloc(&L.d_out, (size_t)out_cap * kResultSlot) != cudaSuccess) return false;
    if (cudaMallocHost(&L.h_status, (size_t)out_cap * sizeof(int)) != cudaSuccess) return false;
    if (cudaMalloc(&L.d_status, (size_t)out_cap * sizeof(int)) != cudaSuccess) return false;
    return true;
}

void lane_free(Lane& L) {
    for (auto& p : L.plans)
        if (p) { perm_plan_destroy(p); p = nullptr; }
    if (L.ext_ws) cudaFree(L.ext_ws);
    if (L.d_in) cudaFree(L.d_in);
    if (L.d_out) cudaFree(L.d_out);
    if (L.d_status) cudaFree(L.d_status);
    if (L.h_in) cudaFreeHost(L.h_in);
    if (L.h_out) cudaFreeHost(L.h_out);
    if (L.h_status) cudaFreeHost(L.h_status);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
    L.stream = nullptr; L.done = nullptr; L.ext_ws = nullptr; L.d_in = nullptr; L.d_out = nullptr;
    L.d_status = nullptr; L.h_in = nullptr; L.h_out = nullptr; L.h_status = nullptr;
    L.inflight.clear();
    L.inflight_at.clear();
    L.busy = false;
}

perm_plan_t lane_plan(perm_server_t s, Lane& L, int dtype, bool large) {
    const int k = dtype_slot(dtype);
    if (!L.plans[k]) {
        perm_opts o = s->opts;
        o.flags = dtype == PERM_C128 ? 0u : (s->opts.flags & PERM_FLAG_WIDE);
        o.method = L.method;
        o.max_batch = large ? 1 : kLaneBatch;
        if (!large) o.mem_budget_bytes = 0;   // the table budget applies to the large lane
        perm_plan_t p = nullptr;
        perm_status st;
        if (large && L.ext_ws)
            st = plan_create_impl(L.n_max, (perm_dtype)dtype, &o, L.ext_ws, L.ext_ws_bytes, &p);
        else
            st = plan_create_impl(L.n_max, (perm_dtype)dtype, &o, nullptr, 0, &p);
        if (st != PERM_OK) return nullptr;
        L.plans[k] = p;
    }
    return L.plans[k];
}

// Launch the requests `batch` (all of one lane) on the lane's stream.
bool lane_launch(perm_server_t s, Lane& L, std::vector<Request*>& batch, bool large) {
    // group by dtype: one perm_batch per dtype, inputs packed per group; each group's
    // results are packed at its own slot size (16 B, or 32 B for wide integers)
    size_t off = 0, out_off = 0;
    int outpos = 0;
    L.inflight.clear();
    L.inflight_at.clear();
    for (int slot = 0; slot < 3; slot++) {
        const int dtype = slot == 0 ? PERM_C128 : (slot == 1 ? PERM_U01 : PERM_I64);
        const size_t rbytes = (dtype != PERM_C128 && (s->opts.flags & PERM_FLAG_WIDE)) ? 32 : 16;
        std::vector<int> sizes;
        const size_t start = off;
        const size_t out_start = out_off;
        const int status_start = outpos;
        for (Request* r : batch) {
            if (r->dtype != dtype) continue;
            std::memcpy(L.h_in + off, r->mat.data(), r->mat.size());
            off += r->mat.size();
            sizes.push_back(r->n);
            r->result_bytes = (int)rbytes;
            L.inflight.push_back(r);
            L.inflight_at.push_back(out_off);
            out_off += rbytes;
            outpos++;
        }
        if (sizes.empty()) continue;
        perm_plan_t p = lane_plan(s, L, dtype, large);
        if (!p) return false;
        if (cudaMemcpyAsync(L.d_in + start, L.h_in + start, off - start, cudaMemcpyHostToDevice,
                            L.stream) != cudaSuccess)
            return false;
        if (perm_batch(p, L.d_in + start, sizes.data(), (int)sizes.size(), L.d_out + out_start,
                       L.d_status + status_start, L.stream) != PERM_OK)
            return false;
    }
    // results back in the same order (dtype groups)
    if (cudaMemcpyAsync(L.h_out, L.d_out, out_off, cudaMemcpyDeviceToHost, L.stream) != cudaSuccess)
        return false;
    if (cudaMemcpyAsync(L.h_status, L.d_status, (size_t)outpos * sizeof(int), cudaMemcpyDeviceToHost,
                        L.stream) != cudaSuccess)
        return false;
    if (cudaEventRecord(L.done, L.stream) != cudaSuccess) return false;
    for (Request* r : batch) r->state.store(1, std::memory_order_relaxed);
    L.busy = true;
    return true;
}

void lane_complete(Lane& L) {
    for (size_t i = 0; i < L.inflight.size(); i++) {
        Request* r = L.inflight[i];
        std::memcpy(r->result, L.h_out + L.inflight_at[i], (size_t)r->result_bytes);
        r->status = L.h_status[i];
        r->state.store(2, std::memory_order_release);
    }
    L.inflight.clear();
    L.inflight_at.clear();
    L.busy = false;
}

void worker_loop(perm_server_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<Request*> batch;
    while (true) {
        if (s->abandon.load()) break;
        bool did = false;
        // completions
        for (int li = 0; li < 3; li++) {
            Lane& L = s->lanes[li];
            if (L.busy) {
                const cudaError_t q = cudaEventQuery(L.done);
                if (q == cudaSuccess) { lane_complete(L); did = true; }
                else if (q != cudaErrorNotReady) { s->failed = true; }
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
        // new batches
        for (int li = 0; li < 3; li++) {
            Lane& L = s->lanes[li];
            if (L.busy || s->failed) continue;
            batch.clear();
            {
                std::lock_guard<std::mutex> g(s->mu);
                auto& q = s->queues[li];
                size_t bytes = 0;
                const size_t max_items = li == 0 ? (size_t)kLaneBatch : 1;
                while (!q.empty() && batch.size() < max_items) {
                    Request* r = q.front();
                    if (bytes + r->mat.size() > L.in_cap) break;
                    bytes += r->mat.size();
                    batch.push_back(r);
                    q.pop_front();
                }
                s->queued -= (int)batch.size();
            }
            if (!batch.empty()) {
                if (!lane_launch(s, L, batch, li != 0)) {
                    s->failed = true;
                    for (Request* r : batch) { r->status = PERM_ECUDA; r->state.store(2, std::memory_order_release); }
                }
                did = true;
            }
        }
        const bool idle = !s->lanes[0].busy && !s->lanes[1].busy && !s->lanes[2].busy;
        if (s->stop.load() && idle) {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->queues[0].empty() && s->queues[1].empty() && s->queues[2].empty()) break;
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
    (void)stream;   // the server owns one stream per lane
    if (!out) return PERM_EINVAL;
    *out = nullptr;
    perm_server_t s = new (std::nothrow) perm_server_s();
    if (!s) return PERM_ENOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.max_batch > 0) s->queue_cap = s->opts.max_batch;
    // table budget for the large lane: default 20 GB (or what is free)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; return PERM_ECUDA; }
    s->table_budget = s->opts.mem_budget_bytes ? s->opts.mem_budget_bytes
                                               : std::min<size_t>((size_t)80 << 30, free_b / 3);
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    Lane& small = s->lanes[0];
    Lane& large = s->lanes[1];
    Lane& ryser = s->lanes[2];
    small.n_max = kSmallN;
    small.priority = greatest;
    large.n_max = kMaxNSZ;
    large.priority = (least + greatest) / 2;
    ryser.n_max = kMaxN;
    ryser.priority = least;
    ryser.method = PERM_METHOD_RYSER;
    bool ok = lane_alloc(small, (size_t)kLaneBatch * kSmallN * kSmallN * 16, kLaneBatch) &&
              lane_alloc(large, (size_t)kMaxN * kMaxN * 16, 1) &&
              lane_alloc(ryser, (size_t)kMaxN * kMaxN * 16, 1);
    if (ok) {
        large.ext_ws_bytes = s->table_budget;
        ok = cudaMalloc(&large.ext_ws, large.ext_ws_bytes) == cudaSuccess;
    }
    // every lane's plans now (they load their kernels): creating one, or loading a kernel,
    // while another lane's work runs could wait for that work
    for (int dt : {PERM_C128, PERM_U01, PERM_I64}) {
        if (ok) ok = lane_plan(s, small, dt, false) != nullptr;
        if (ok) ok = lane_plan(s, ryser, dt, true) != nullptr;
    }
    if (ok) ok = lane_plan(s, large, PERM_C128, true) != nullptr;   // the table lane takes complex requests
    if (!ok) {
        cudaGetLastError();
        for (auto& L : s->lanes) lane_free(L);
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
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->queued >= s->queue_cap) return PERM_EAGAIN;
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        Request* raw = r.get();
        int lane = 0;
        if (n > kSmallN) {
            // complex: admission by table memory, Store-zechin if its chains fit the budget,
            // else Ryser; integers: Ryser (the method PERM_METHOD_AUTO picks for them)
            const bool fits = auto_uses_sz(dtype) && n <= kMaxNSZ &&
                              sz_matrix_workspace_bytes(dtype, n, kLargeLow) + ((size_t)1 << 20) <= s->table_budget;
            lane = fits ? 1 : 2;
        }
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
            busy = s->lanes[0].busy || s->lanes[1].busy || s->lanes[2].busy || !s->queues[0].empty() ||
                   !s->queues[1].empty() || !s->queues[2].empty();
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
    delete s;
    return result;
}

}  // extern "C"
