// api.cu -- the C ABI of libperm: plans, batched evaluation, status strings,
// and the FP64 peak measurement used as a roofline denominator.
//
// perm_batch (Su & Zheng, arXiv:1802.02779: Store-zechin, Section 4; Ryser,
// Section 3.3) classifies every matrix by order and method, uploads one
// descriptor array, and enqueues on the caller's stream:
//   - n = 0           -> per = 1
//   - Store-zechin    -> one persistent launch for all matrices whose chain
//                        workspace fits one CTA slice (one CTA per matrix),
//                        larger ones one at a time over the whole GPU
//   - Ryser           -> one launch per distinct order (plus a finishing kernel)
// PERM_METHOD_AUTO sends complex matrices to Store-zechin where its tables
// fit and integer matrices to Ryser (auto_uses_sz, with the measurements).
// The method per matrix depends only on (n, dtype) and the plan, so a matrix
// gives bit-identical results alone or in any batch.
#include "perm_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

using namespace perm;

constexpr size_t kGraphCacheCap = 16;

// One captured batch (PERM_FLAG_GRAPH): its launch sequence as a CUDA graph.
struct GraphEntry {
    unsigned long long key = 0;
    int count = 0;
    std::vector<int> sizes;
    const void* mats = nullptr;
    const void* out = nullptr;
    const int* status = nullptr;
    ItemDesc* desc = nullptr;          // device copy of the descriptors the graph reads
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (desc) cudaFree(desc);
        exec = nullptr; graph = nullptr; desc = nullptr;
    }
};

struct perm_plan_s {
    int device = 0;
    int n_max = 0;
    int dtype = PERM_C128;
    int method = PERM_METHOD_AUTO;
    unsigned flags = 0;
    int max_batch = 65536;
    int num_sms = 0;
    int m_low = 12;               // chain width of the batched kernel (two CTAs per SM)
    // layer path (matrices over the whole GPU, one launch per layer): orders above
    // kLayerSmallN, and (the *_small fields) orders up to it
    int m_single = 13;            // chain width
    int layer_threads = 512;      // CTA size of the complex kernel (384: two CTAs per SM)
    int layer_grid_mult = 1;      // CTAs per launch, in units of the SM count
    int m_small = 12;
    int layer_threads_small = 384;
    int layer_grid_small = 2;
    int m_few = 0;                // orders up to kLayerSmallN, at most kFlowMaxCount matrices:
                                  // 0 = by order and count (sz_layer_default_shape), else this
    bool tail_to_layers = true;   // the batched kernel's last partial round takes the layer path
    int flow = -1;                // complex orders <= kLayerSmallN, the dataflow layer launch:
                                  // 1 always, 0 never, -1 for at most kFlowMaxCount matrices
    int c128_threads = 384;       // CTA size of the batched complex kernel
    int int_threads = 256;        // CTA size of the batched integer kernel
    int out_words = 2;            // integer result slot in 64-bit words (4 with PERM_FLAG_WIDE)
    size_t budget = 0;

    // Store-zechin
    int sz_batch_nmax = 0;        // largest n that runs one-CTA-per-matrix
    int sz_grid = 0;              // persistent CTAs of the batched kernel
    size_t sz_ws_per_cta = 0;
    int sz_single_nmax = 0;       // largest n that runs at all with Store-zechin
    void* ws = nullptr;
    size_t ws_bytes = 0;

    // Ryser
    void* partials = nullptr;
    size_t partials_bytes = 0;
    long long partials_cap = 0;   // in parts

    // descriptors: pinned host staging + device copy
    unsigned char* h_stage = nullptr;
    unsigned char* d_stage = nullptr;
    size_t stage_bytes = 0;
    cudaEvent_t stage_free = nullptr;
    unsigned* d_counter = nullptr;
    int* d_widths = nullptr;      // integer Ryser: width and row-sum class per matrix of a launch

    bool ext_ws = false;          // workspace owned by someone else (the server)

    // host-buffer path
    void* d_in = nullptr;
    size_t d_in_bytes = 0;
    void* d_out = nullptr;
    int* d_status = nullptr;

    bool tuned = false;           // chosen by the autotuner

    // graph cache (PERM_FLAG_GRAPH)
    std::vector<GraphEntry> graphs;
    unsigned long long graph_clock = 0;
};

namespace {

size_t elem_bytes(int dtype) { return dtype == PERM_C128 ? 16 : 8; }

bool valid_dtype(int d) { return d == PERM_C128 || d == PERM_U01 || d == PERM_I64; }

template <class T>
void release(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

perm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PERM_OK : PERM_ECUDA; }

int sz_batch_limit(perm_plan_t p, int complex_cap = 20) {
    // One CTA per matrix when the per-CTA chain workspace stays <= 80 MB.  For complex
    // matrices at most n = 20: measured on GB300 (batches of 512-4096 matrices), the layer
    // path, with every same-order matrix in each layer launch, is 3-11% faster at n = 21-22,
    // where a batch leaves the one-CTA-per-matrix kernel a long last wave; the batched kernel
    // is 4-8% faster up to n = 19.  Both give the same bits.
    int best = 0;
    for (int n = 1; n <= std::min(p->n_max, kMaxNSZ); n++) {
        if (sz_matrix_workspace_bytes(p->dtype, n, p->m_low) <= (size_t)80 << 20) best = n;
    }
    if (p->dtype == PERM_C128) best = std::min(best, complex_cap);
    return best;
}

// Chain width of the layer path for order n, with `count` matrices of that order in a launch
// (the default: more than kFlowMaxCount).
int layer_m(perm_plan_t p, int n, int count = kFlowMaxCount + 1) {
    if (n > kLayerSmallN) return p->m_single;
    if (count > kFlowMaxCount || p->dtype != PERM_C128) return p->m_small;
    if (p->m_few) return p->m_few;
    int m = 0, threads = 0;
    sz_layer_default_shape(n, count, &m, &threads);
    return m;
}

}  // namespace

// Plan creation with an optional caller-owned Store-zechin workspace.
perm_status plan_create_impl(int n_max, perm_dtype dtype, const perm_opts* opts, void* ext_ws,
                             size_t ext_ws_bytes, perm_plan_t* out);
static perm_status plan_create_tuned(int n_max, perm_dtype dtype, const perm_opts* opts,
                                     perm_plan_t* out);
// Kernel-shape choices of the autotuner (0 = default).
struct PlanShape {
    int m_low = 0;           // chain width of the batched kernel
    int threads = 0;         // CTA size of the batched kernel
    int batch_nmax = -1;     // largest complex order of the batched kernel (-1: 20)
    int layer_threads = 0;   // layer path, complex orders <= kLayerSmallN: CTA size (384 or 512),
    int m_single = 0;        // chain width,
    int layer_grid_mult = 0; // and CTAs per layer launch in units of the SM count
};
static perm_status plan_create_core(int n_max, perm_dtype dtype, const perm_opts* opts, void* ext_ws,
                                    size_t ext_ws_bytes, PlanShape shape, perm_plan_t* out);

extern "C" {

const char* perm_strerror(perm_status s) {
    switch (s) {
        case PERM_OK: return "ok";
        case PERM_EINVAL: return "invalid argument";
        case PERM_ENOMEM: return "workspace does not fit the memory budget";
        case PERM_EOVERFLOW: return "integer permanent bound exceeds the result width (2^128; 2^192 with PERM_FLAG_WIDE)";
        case PERM_ECUDA: return "CUDA runtime error";
        case PERM_EAGAIN: return "try again";
        case PERM_ETIMEDOUT: return "timed out";
        case PERM_ESHUTDOWN: return "shutting down";
        case PERM_ENOTFOUND: return "unknown ticket";
    }
    return "unknown status";
}

const char* perm_version(void) { return "0.1.0"; }

perm_status perm_plan_create(int n_max, perm_dtype dtype, const perm_opts* opts, perm_plan_t* out) {
    if (opts && (opts->flags & PERM_FLAG_AUTOTUNE)) return plan_create_tuned(n_max, dtype, opts, out);
    return plan_create_impl(n_max, dtype, opts, nullptr, 0, out);
}

}  // extern "C"

perm_status plan_create_impl(int n_max, perm_dtype dtype, const perm_opts* opts, void* ext_ws,
                             size_t ext_ws_bytes, perm_plan_t* out) {
    return plan_create_core(n_max, dtype, opts, ext_ws, ext_ws_bytes, PlanShape{}, out);
}

static perm_status plan_create_core(int n_max, perm_dtype dtype, const perm_opts* opts, void* ext_ws,
                                    size_t ext_ws_bytes, PlanShape shape, perm_plan_t* out) {
    if (!out) return PERM_EINVAL;
    *out = nullptr;
    if (n_max < 0 || n_max > kMaxN || !valid_dtype(dtype)) return PERM_EINVAL;
    perm_opts o{};
    if (opts) o = *opts;
    if (o.method < PERM_METHOD_AUTO || o.method > PERM_METHOD_RYSER) return PERM_EINVAL;
    if (o.max_batch < 0 || o.ctas_per_sm < 0 || o.low_cols < 0 || o.low_cols > kMaxLow)
        return PERM_EINVAL;
    if (o.method == PERM_METHOD_SZ && n_max > kMaxNSZ) return PERM_EINVAL;
    if ((o.flags & PERM_FLAG_WIDE) && dtype == PERM_C128) return PERM_EINVAL;

    perm_plan_t p = new (std::nothrow) perm_plan_s();
    if (!p) return PERM_ENOMEM;
    p->n_max = n_max;
    p->dtype = dtype;
    p->method = o.method;
    p->flags = o.flags;
    p->out_words = (o.flags & PERM_FLAG_WIDE) ? 4 : 2;
    p->max_batch = o.max_batch ? o.max_batch : 65536;
    p->m_low = o.low_cols ? o.low_cols : 12;
    sz_layer_default_shape(kLayerSmallN + 1, kFlowMaxCount + 1, &p->m_single, &p->layer_threads);
    sz_layer_default_shape(kLayerSmallN, kFlowMaxCount + 1, &p->m_small, &p->layer_threads_small);
    if (dtype != PERM_C128) p->m_small = p->m_single;   // integers: one shape (the 256-thread kernel)
    if (o.low_cols) p->m_single = p->m_small = p->m_few = o.low_cols;
    if (shape.m_single >= 1 && shape.m_single <= kMaxLow && !o.low_cols) p->m_small = shape.m_single;
    if (shape.layer_threads == 384 || shape.layer_threads == 512 || shape.layer_threads == 768)
        p->layer_threads_small = shape.layer_threads;
    if (shape.layer_grid_mult >= 1 && shape.layer_grid_mult <= 8) p->layer_grid_small = shape.layer_grid_mult;
    // experiment knobs (results are bit-identical for every choice)
    if (const char* v = getenv("LIBPERM_SZ_LOW")) { int x = atoi(v); if (x >= 1 && x <= kMaxLow) p->m_low = x; }
    if (const char* v = getenv("LIBPERM_SZ_THREADS")) {
        const int x = atoi(v);
        if (sz_c128_threads_valid(x)) p->c128_threads = x;
        if (sz_int_threads_valid(x)) p->int_threads = x;
    }
    if (const char* v = getenv("LIBPERM_SZ_TAIL_LAYERS")) p->tail_to_layers = atoi(v) != 0;
    if (const char* v = getenv("LIBPERM_SZ_FLOW")) p->flow = atoi(v) != 0 ? 1 : 0;
    if (const char* v = getenv("LIBPERM_SZ_LAYER_THREADS")) {
        const int x = atoi(v);
        if (x == 384 || x == 512 || x == 768) p->layer_threads = p->layer_threads_small = x;
    }
    if (const char* v = getenv("LIBPERM_SZ_LAYER_GRID")) {
        const int x = atoi(v);
        if (x >= 1 && x <= 8) p->layer_grid_mult = p->layer_grid_small = x;
    }
    if (shape.m_low >= 1 && shape.m_low <= kMaxLow) p->m_low = shape.m_low;
    if (dtype == PERM_C128 && sz_c128_threads_valid(shape.threads)) p->c128_threads = shape.threads;
    if (dtype != PERM_C128 && sz_int_threads_valid(shape.threads)) p->int_threads = shape.threads;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) { delete p; return PERM_ECUDA; }
    p->budget = o.mem_budget_bytes ? o.mem_budget_bytes : (size_t)(0.45 * (double)free_b);
    if (ext_ws) p->budget = ext_ws_bytes;

    // ---- Store-zechin workspace ----
    size_t sz_batched = 0, sz_single = 0;
    const bool uses_sz = p->method == PERM_METHOD_SZ || (p->method == PERM_METHOD_AUTO && auto_uses_sz(dtype));
    if (uses_sz && n_max >= 1) {
        p->sz_batch_nmax = sz_batch_limit(p, shape.batch_nmax >= 0 ? shape.batch_nmax : 20);
        // The workspace is sized for the batched kernel at its default largest order (or the tuned
        // one, if larger) even when a smaller order is chosen: the layer path then shares the same
        // workspace among the matrices of one order, as many as it holds.
        const int ws_nmax = std::max(p->sz_batch_nmax, sz_batch_limit(p, 20));
        // experiment knob: largest order of the one-CTA-per-matrix kernel (the others take the
        // layer path; both give the same bits)
        if (const char* v = getenv("LIBPERM_SZ_BATCH_NMAX")) {
            const int x = atoi(v);
            if (x >= 0 && x < p->sz_batch_nmax) p->sz_batch_nmax = x;
        }
        p->sz_ws_per_cta = sz_matrix_workspace_bytes(dtype, ws_nmax, p->m_low);
        if (sz_init_tables() != cudaSuccess) { delete p; return PERM_ECUDA; }
        int per_sm = o.ctas_per_sm ? o.ctas_per_sm
                                   : sz_batched_occupancy(dtype, std::max(1, ws_nmax), p->m_low,
                                                          dtype == PERM_C128 ? p->c128_threads : p->int_threads);
        p->sz_grid = p->num_sms * per_sm;
        sz_batched = p->sz_ws_per_cta * (size_t)p->sz_grid;
        // largest n whose single-matrix workspace fits the remaining budget
        for (int n = 1; n <= std::min(n_max, kMaxNSZ); n++) {
            size_t need = 0;
            for (int c = 1; c <= kFlowMaxCount + 1; c++)
                need = std::max(need, sz_matrix_workspace_bytes(dtype, n, layer_m(p, n, c)));
            if (need + (size_t)(1 << 20) <= p->budget) {
                p->sz_single_nmax = n;
                sz_single = std::max(sz_single, need);
            }
        }
        if (sz_batched > p->budget) {   // shrink the persistent grid to the budget
            p->sz_grid = (int)std::max<size_t>(1, p->budget / std::max<size_t>(1, p->sz_ws_per_cta));
            sz_batched = p->sz_ws_per_cta * (size_t)p->sz_grid;
        }
        if (p->method == PERM_METHOD_SZ && p->sz_single_nmax < std::min(n_max, kMaxNSZ)) {
            delete p;
            return PERM_ENOMEM;
        }
    }
    p->ws_bytes = std::max(sz_batched, sz_single);

    // load every kernel this plan can launch now, not at its first launch
    if ((uses_sz && sz_preload(dtype) != cudaSuccess) || ryser_preload(dtype, n_max) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return PERM_ECUDA;
    }

    // ---- Ryser partials (32-40 B per piece of codes): one matrix of the largest order,
    // max_batch matrices of one piece each, and up to 2^20 pieces (32-40 MB) so that a batch
    // of mid-size matrices fills the GPU in one launch instead of many small ones ----
    long long max_parts = 1;
    for (int n = 1; n <= n_max; n++) max_parts = std::max(max_parts, ryser_parts(dtype, n));
    long long cap = std::max<long long>(max_parts, (long long)p->max_batch);
    cap = std::max<long long>(cap, std::min<long long>(max_parts * (long long)p->max_batch, 1ll << 20));
    p->partials_cap = cap;
    p->partials_bytes = (size_t)cap * ryser_partial_bytes(dtype);

    // ---- descriptor staging ----
    const int mb = p->max_batch;
    p->stage_bytes = (size_t)mb * sizeof(ItemDesc) + 256;

    e = cudaSuccess;
    if (ext_ws) {
        if (p->ws_bytes > ext_ws_bytes) { delete p; return PERM_ENOMEM; }
        p->ws = ext_ws;
        p->ext_ws = true;
    } else if (p->ws_bytes) {
        e = cudaMalloc(&p->ws, p->ws_bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->partials, p->partials_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_stage, p->stage_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_stage, p->stage_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_counter, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_widths, 2 * (size_t)p->max_batch * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->stage_free, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        perm_plan_destroy(p);
        return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
    }
    *out = p;
    return PERM_OK;
}

extern "C" {

perm_status perm_plan_destroy(perm_plan_t p) {
    if (!p) return PERM_OK;
    cudaDeviceSynchronize();
    for (auto& g : p->graphs) g.release();
    p->graphs.clear();
    if (p->ext_ws) p->ws = nullptr;
    release(p->ws);
    release(p->partials);
    release(p->d_stage);
    release(p->d_counter);
    release(p->d_widths);
    release(p->d_in);
    release(p->d_out);
    release(p->d_status);
    if (p->h_stage) cudaFreeHost(p->h_stage);
    if (p->stage_free) cudaEventDestroy(p->stage_free);
    delete p;
    return PERM_OK;
}

int perm_plan_describe(perm_plan_t p, char* buf, size_t len) {
    if (!p) return -1;
    const char* dt = p->dtype == PERM_C128 ? "c128" : (p->dtype == PERM_U01 ? "u01" : "i64");
    return snprintf(buf, len,
                    "{\"dtype\": \"%s\", \"n_max\": %d, \"method\": %d, \"flags\": %u, "
                    "\"sz_batch_nmax\": %d, \"sz_single_nmax\": %d, \"chain_width_batched\": %d, "
                    "\"chain_width_single\": %d, \"cta_threads\": %d, \"batched_grid\": %d, "
                    "\"layer_cta_threads\": %d, \"layer_ctas_per_sm\": %d, \"layer_small_nmax\": %d, "
                    "\"chain_width_layer_few\": %d, \"chain_width_layer_few_n20\": %d, "
                    "\"chain_width_layer_small\": %d, \"layer_cta_threads_small\": %d, "
                    "\"layer_ctas_per_sm_small\": %d, "
                    "\"workspace_bytes\": %zu, \"out_words\": %d, \"autotuned\": %s}",
                    dt, p->n_max, p->method, p->flags, p->sz_batch_nmax, p->sz_single_nmax, p->m_low,
                    p->m_single, p->dtype == PERM_C128 ? p->c128_threads : p->int_threads, p->sz_grid,
                    p->dtype == PERM_C128 ? p->layer_threads : 256, p->layer_grid_mult, kLayerSmallN,
                    layer_m(p, kLayerSmallN, 1), layer_m(p, 20, 1),
                    p->m_small, p->dtype == PERM_C128 ? p->layer_threads_small : 256, p->layer_grid_small,
                    perm_plan_workspace_bytes(p), p->dtype == PERM_C128 ? 0 : p->out_words,
                    p->tuned ? "true" : "false");
}

size_t perm_plan_workspace_bytes(perm_plan_t p) {
    return p ? p->ws_bytes + p->partials_bytes + p->stage_bytes + p->d_in_bytes : 0;
}

}  // extern "C"

namespace {

// Classification of one batch: descriptors in launch order and the launch list.
struct BatchLayout {
    std::vector<ItemDesc> desc;      // [n = 0][batched Store-zechin][Store-zechin by n][Ryser by n]
    size_t triv_at = 0, ntriv = 0;
    size_t szb_at = 0, nszb = 0;
    int szb_nmax = 0;
    struct Group { int n; size_t at; int cnt; };
    std::vector<Group> szs;          // one-matrix-over-the-GPU Store-zechin, by order
    std::vector<Group> ry;
};

perm_status classify(perm_plan_t p, const int* sizes, int count, BatchLayout& L) {
    const bool plain = (p->flags & PERM_FLAG_PLAIN) != 0;
    std::vector<ItemDesc> triv, szb;
    std::map<int, std::vector<ItemDesc>> ry;   // by n, ascending
    std::map<int, std::vector<ItemDesc>> szs;  // by n, ascending
    long long off = 0;
    for (int i = 0; i < count; i++) {
        const int n = sizes[i];
        ItemDesc d{off, n, i};
        off += (long long)n * n;
        if (n == 0) { triv.push_back(d); continue; }
        bool use_sz = false;
        if (p->method == PERM_METHOD_SZ) {
            if (n > p->sz_single_nmax) return PERM_ENOMEM;
            use_sz = true;
        } else if (p->method == PERM_METHOD_AUTO) {
            use_sz = auto_uses_sz(p->dtype) && n <= p->sz_single_nmax;
        }
        if (use_sz) {
            if (!plain && n <= p->sz_batch_nmax) szb.push_back(d);
            else szs[n].push_back(d);
        } else {
            ry[n].push_back(d);
        }
    }
    // With fewer such matrices than SMs, one CTA per matrix would leave most of the GPU idle
    // (and one n = 20 matrix takes ~20 ms on one CTA): the layer path spreads every matrix's
    // chains over the whole GPU instead.  Both paths sum every entry in the same order, so
    // the results are the same bits.
    if (!plain && (int)szb.size() < p->num_sms) {
        for (auto& d : szb) szs[d.n].push_back(d);
        szb.clear();
    }
    // longest matrices first for the persistent queue
    std::stable_sort(szb.begin(), szb.end(), [](const ItemDesc& a, const ItemDesc& b) { return a.n > b.n; });
    // The persistent grid takes the matrices in rounds of one per CTA; a last, partial round
    // would leave the other CTAs idle for a whole matrix's time.  Complex matrices of that round
    // (the shortest, at the end of the queue) take the layer path instead, which spreads their
    // chains over every SM after the batched launch.  Same bits either way.
    if (!plain && p->dtype == PERM_C128 && p->tail_to_layers && (int)szb.size() > p->sz_grid) {
        const size_t rem = szb.size() % (size_t)p->sz_grid;
        for (size_t i = szb.size() - rem; i < szb.size(); i++) szs[szb[i].n].push_back(szb[i]);
        szb.resize(szb.size() - rem);
    }
    L.triv_at = L.desc.size();
    L.ntriv = triv.size();
    L.desc.insert(L.desc.end(), triv.begin(), triv.end());
    L.szb_at = L.desc.size();
    L.nszb = szb.size();
    L.szb_nmax = szb.empty() ? 0 : szb.front().n;
    L.desc.insert(L.desc.end(), szb.begin(), szb.end());
    for (auto& kv : szs) {
        L.szs.push_back({kv.first, L.desc.size(), (int)kv.second.size()});
        L.desc.insert(L.desc.end(), kv.second.begin(), kv.second.end());
    }
    for (auto& kv : ry) {
        L.ry.push_back({kv.first, L.desc.size(), (int)kv.second.size()});
        L.desc.insert(L.desc.end(), kv.second.begin(), kv.second.end());
    }
    return PERM_OK;
}

// Enqueue every launch of a classified batch on `st` (descriptors at `dd` on the device).
perm_status enqueue(perm_plan_t p, const BatchLayout& L, const void* mats, const ItemDesc* dd,
                    void* out, int* item_status, cudaStream_t st) {
    const bool plain = (p->flags & PERM_FLAG_PLAIN) != 0;
    cudaError_t e;
    if (L.ntriv) {
        e = launch_trivial(p->dtype, dd + L.triv_at, (int)L.ntriv, out, p->out_words, item_status, st);
        if (e != cudaSuccess) return PERM_ECUDA;
    }
    if (L.nszb) {
        e = cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return PERM_ECUDA;
        const int grid = std::min<int>(p->sz_grid, (int)L.nszb);
        e = sz_launch_batched(p->dtype, mats, dd + L.szb_at, (int)L.nszb, L.szb_nmax, p->m_low,
                              p->dtype == PERM_C128 ? p->c128_threads : p->int_threads, out, p->out_words,
                              item_status, p->ws, p->sz_ws_per_cta, grid, p->d_counter, st);
        if (e != cudaSuccess) return PERM_ECUDA;
    }
    for (auto& g : L.szs) {
        // matrices of one order share every layer launch, as many as the workspace holds
        // (one at a time when plain): the small first and last layers of one matrix leave
        // most of the GPU idle, several fill it.  Two CTAs' worth of chains per SM and
        // layer amortise the per-CTA set-up, and every layer is its own launch, which gives
        // the scheduler a point to interleave work from higher-priority streams.
        int lm = layer_m(p, g.n, plain ? 1 : g.cnt);
        const bool small = g.n <= kLayerSmallN;
        size_t ws_item = sz_matrix_workspace_bytes(p->dtype, g.n, lm);
        if (ws_item > p->ws_bytes) {           // the workspace was sized for the batch shape
            lm = layer_m(p, g.n);
            ws_item = sz_matrix_workspace_bytes(p->dtype, g.n, lm);
        }
        // complex orders up to kLayerSmallN, a few matrices: every layer in one dataflow launch,
        // whose chains start as their predecessors finish (measured on GB300: one n = 22 matrix
        // 0.71 ms against 0.86 ms in layer launches, four 1.62 against 1.80 ms; with 16 or more
        // matrices the layer launches are already full and the two are within 3 %)
        const size_t ws_flow = sz_flow_workspace_bytes(g.n, lm);
        const bool want_flow = p->flow == 1 || (p->flow < 0 && (plain || g.cnt <= kFlowMaxCount));
        const bool flow = want_flow && small && p->dtype == PERM_C128 && ws_flow <= p->ws_bytes;
        if (flow) ws_item = ws_flow;
        long long per_launch = ws_item ? (long long)(p->ws_bytes / ws_item) : (long long)g.cnt;
        per_launch = std::max<long long>(1, per_launch);
        if (plain) per_launch = 1;
        for (int b0 = 0; b0 < g.cnt; b0 += (int)per_launch) {
            const int c = (int)std::min<long long>(per_launch, g.cnt - b0);
            if (flow)
                e = sz_launch_flow(mats, dd + g.at + b0, c, g.n, lm, out, item_status, p->ws, ws_item,
                                   p->d_counter + 1, p->num_sms, st);
            else
                e = sz_launch_layers(p->dtype, mats, dd + g.at + b0, c, g.n, lm, out, p->out_words, item_status,
                                     p->ws, ws_item, (small ? p->layer_grid_small : p->layer_grid_mult) * p->num_sms,
                                     st, small ? p->layer_threads_small : p->layer_threads);
            if (e != cudaSuccess) return PERM_ECUDA;
        }
    }
    for (auto& g : L.ry) {
        const long long parts = ryser_parts(p->dtype, g.n);
        // matrices per launch limited by the partials buffer (and one per launch when plain)
        long long per_launch = std::max<long long>(1, p->partials_cap / parts);
        if (plain) per_launch = 1;
        for (int b0 = 0; b0 < g.cnt; b0 += (int)per_launch) {
            const int c = (int)std::min<long long>(per_launch, g.cnt - b0);
            e = ryser_launch_group(p->dtype, g.n, mats, dd + g.at + b0, c, p->partials, p->d_widths,
                                   out, p->out_words, p->out_words == 4, item_status, 1 << 30, st);
            if (e != cudaSuccess) return PERM_ECUDA;
        }
    }
    return PERM_OK;
}

unsigned long long batch_key(const void* mats, const int* sizes, int count, const void* out,
                             const int* item_status) {
    // FNV-1a over the shape and the buffer addresses
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&h](unsigned long long v) {
        for (int b = 0; b < 8; b++) { h ^= (v >> (8 * b)) & 0xff; h *= 1099511628211ull; }
    };
    mix((unsigned long long)(uintptr_t)mats);
    mix((unsigned long long)(uintptr_t)out);
    mix((unsigned long long)(uintptr_t)item_status);
    mix((unsigned long long)count);
    for (int i = 0; i < count; i++) mix((unsigned long long)sizes[i]);
    return h;
}

perm_status batch_graph(perm_plan_t p, const void* mats, const int* sizes, int count, void* out,
                        int* item_status, cudaStream_t st) {
    const unsigned long long key = batch_key(mats, sizes, count, out, item_status);
    for (auto& g : p->graphs) {
        if (g.key == key && g.count == count && g.sizes == std::vector<int>(sizes, sizes + count) &&
            g.mats == mats && g.out == out && g.status == item_status) {
            g.last_use = ++p->graph_clock;
            return cudaGraphLaunch(g.exec, st) == cudaSuccess ? PERM_OK : PERM_ECUDA;
        }
    }
    BatchLayout L;
    perm_status ps = classify(p, sizes, count, L);
    if (ps != PERM_OK) return ps;
    GraphEntry g;
    g.key = key;
    g.count = count;
    g.sizes.assign(sizes, sizes + count);
    g.mats = mats;
    g.out = out;
    g.status = item_status;
    const size_t bytes = std::max<size_t>(1, L.desc.size()) * sizeof(ItemDesc);
    if (cudaMalloc(&g.desc, bytes) != cudaSuccess) { cudaGetLastError(); return PERM_ENOMEM; }
    cudaError_t e = cudaMemcpy(g.desc, L.desc.data(), L.desc.size() * sizeof(ItemDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaFree(g.desc); return PERM_ECUDA; }
    ps = enqueue(p, L, mats, g.desc, out, item_status, st);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (ps != PERM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaFree(g.desc);
        cudaGetLastError();
        return ps != PERM_OK ? ps : PERM_ECUDA;
    }
    g.graph = graph;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); cudaFree(g.desc); return PERM_ECUDA; }
    if (p->graphs.size() >= kGraphCacheCap) {   // evict the least recently used graph
        auto it = std::min_element(p->graphs.begin(), p->graphs.end(),
                                   [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
        cudaStreamSynchronize(st);
        it->release();
        p->graphs.erase(it);
    }
    g.last_use = ++p->graph_clock;
    p->graphs.push_back(g);
    return cudaGraphLaunch(g.exec, st) == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

}  // namespace

extern "C" {

perm_status perm_batch(perm_plan_t p, const void* mats, const int* sizes, int count, void* out,
                       int* item_status, void* stream) {
    if (!p || count < 0) return PERM_EINVAL;
    if (count == 0) return PERM_OK;
    if (!sizes || !out || count > p->max_batch) return PERM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    bool any_nonempty = false;
    for (int i = 0; i < count; i++) {
        if (sizes[i] < 0 || sizes[i] > p->n_max) return PERM_EINVAL;
        if (sizes[i] > 0) any_nonempty = true;
    }
    if (any_nonempty && !mats) return PERM_EINVAL;
    if ((p->flags & PERM_FLAG_GRAPH) && st != nullptr)
        return batch_graph(p, mats, sizes, count, out, item_status, st);

    BatchLayout L;
    perm_status ps = classify(p, sizes, count, L);
    if (ps != PERM_OK) return ps;
    const size_t used = L.desc.size() * sizeof(ItemDesc);
    if (used > p->stage_bytes) return PERM_EINVAL;
    cudaError_t e = cudaEventSynchronize(p->stage_free);   // previous upload finished reading
    if (e != cudaSuccess) return PERM_ECUDA;
    if (used) std::memcpy(p->h_stage, L.desc.data(), used);
    if (used) e = cudaMemcpyAsync(p->d_stage, p->h_stage, used, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->stage_free, st);
    if (e != cudaSuccess) return PERM_ECUDA;
    return enqueue(p, L, mats, reinterpret_cast<const ItemDesc*>(p->d_stage), out, item_status, st);
}

perm_status perm_batch_host(perm_plan_t p, const void* mats, const int* sizes, int count, void* out,
                            int* item_status, void* stream) {
    if (!p || count < 0) return PERM_EINVAL;
    if (count == 0) return PERM_OK;
    if (!sizes || !out || count > p->max_batch) return PERM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    size_t elems = 0;
    for (int i = 0; i < count; i++) {
        if (sizes[i] < 0 || sizes[i] > p->n_max) return PERM_EINVAL;
        elems += (size_t)sizes[i] * sizes[i];
    }
    if (elems && !mats) return PERM_EINVAL;
    const size_t in_bytes = elems * elem_bytes(p->dtype);
    cudaError_t e = cudaSuccess;
    if (in_bytes > p->d_in_bytes) {
        // grow-only device staging for the host path
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) { release(p->d_in); p->d_in_bytes = 0; e = cudaMalloc(&p->d_in, in_bytes); }
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
        p->d_in_bytes = in_bytes;
    }
    const size_t out_bytes = p->dtype == PERM_C128 ? 16 : 8 * (size_t)p->out_words;
    if (!p->d_out) {
        e = cudaMalloc(&p->d_out, (size_t)p->max_batch * out_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_status, (size_t)p->max_batch * sizeof(int));
        if (e != cudaSuccess) return PERM_ECUDA;
    }
    if (in_bytes) e = cudaMemcpyAsync(p->d_in, mats, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return PERM_ECUDA;
    perm_status s = perm_batch(p, p->d_in, sizes, count, p->d_out, p->d_status, st);
    if (s != PERM_OK) return s;
    e = cudaMemcpyAsync(out, p->d_out, (size_t)count * out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && item_status)
        e = cudaMemcpyAsync(item_status, p->d_status, (size_t)count * sizeof(int),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// One large matrix split over several GPUs by Ryser's code range (Section 3.3,
// Eq. 4 / Glynn's form).  The codes of an order-n matrix are cut into the
// same pieces perm_batch uses; a rank computes the partial sums of a
// contiguous range of pieces, the ranks' partial sums are gathered in piece
// order, and one finishing call sums all of them in the fixed order
// perm_batch uses.  So the result is the same bits for every number of ranks.
// ---------------------------------------------------------------------------
namespace {

// Upload one descriptor {offset 0, order n, slot 0} through the plan's staging.
perm_status stage_one(perm_plan_t p, int n, cudaStream_t st) {
    const ItemDesc d{0, n, 0};
    cudaError_t e = cudaEventSynchronize(p->stage_free);
    if (e != cudaSuccess) return PERM_ECUDA;
    std::memcpy(p->h_stage, &d, sizeof(d));
    e = cudaMemcpyAsync(p->d_stage, p->h_stage, sizeof(d), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->stage_free, st);
    return cuda_status(e);
}

}  // namespace

extern "C" {

perm_status perm_ryser_pieces(int n, perm_dtype dtype, long long* pieces, size_t* piece_bytes) {
    if (!valid_dtype(dtype) || n < 1 || n > kMaxN || !pieces) return PERM_EINVAL;
    *pieces = ryser_parts(dtype, n);
    if (piece_bytes) *piece_bytes = ryser_partial_bytes(dtype);
    return PERM_OK;
}

perm_status perm_ryser_split(long long pieces, int rank, int world, long long* begin, long long* end) {
    if (pieces < 1 || world < 1 || rank < 0 || rank >= world || !begin || !end) return PERM_EINVAL;
    // balanced contiguous ranges: rank r takes [floor(P r / W), floor(P (r+1) / W)); computed
    // without overflow for P < 2^40 and W < 2^20
    *begin = (long long)((unsigned long long)pieces * (unsigned long long)rank / (unsigned long long)world);
    *end = (long long)((unsigned long long)pieces * (unsigned long long)(rank + 1) / (unsigned long long)world);
    return PERM_OK;
}

perm_status perm_ryser_partials(perm_plan_t p, const void* mat, int n, long long begin, long long end,
                                void* partials, void* stream) {
    if (!p || !mat || !partials || n < 1 || n > p->n_max) return PERM_EINVAL;
    if (begin < 0 || end < begin || end > ryser_parts(p->dtype, n)) return PERM_EINVAL;
    if (begin == end) return PERM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    perm_status ps = stage_one(p, n, st);
    if (ps != PERM_OK) return ps;
    const cudaError_t e = ryser_launch_pieces(p->dtype, n, mat, reinterpret_cast<const ItemDesc*>(p->d_stage),
                                              begin, end, partials, p->d_widths, p->out_words == 4, 1 << 30, st);
    return e == cudaErrorInvalidValue ? PERM_EINVAL : cuda_status(e);
}

perm_status perm_ryser_finish(perm_plan_t p, int n, const void* partials, void* out, int* item_status,
                              void* stream) {
    if (!p || !partials || !out || n < 1 || n > p->n_max) return PERM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    perm_status ps = stage_one(p, n, st);
    if (ps != PERM_OK) return ps;
    const cudaError_t e = ryser_finish_one(p->dtype, n, reinterpret_cast<const ItemDesc*>(p->d_stage), partials,
                                           out, p->out_words, item_status, st);
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner (PERM_FLAG_AUTOTUNE).  Times candidate launch shapes on synthetic
// batches and keeps the fastest of each:
//   1. the batched Store-zechin kernel: CTA size x chain width, at the plan's
//      largest batched order (at most 20);
//   2. complex plans with n_max >= 21: the largest order that still runs one
//      CTA per matrix rather than the layer path (19..22), from batches of
//      2 x SMs matrices per order;
//   3. complex plans with n_max >= 21: the layer path's CTA size, chain width
//      and CTAs per launch for orders up to 24, on one matrix of order
//      min(n_max, 24) (larger orders keep chains of 2^13 at one 512-thread CTA
//      per SM, measured faster at every order from 25 to 32).
// Every choice gives bit-identical results: every entry sums its terms over its
// columns in ascending order whatever the shape.  Choices are cached per
// (device, dtype, n_max) for the process, and in the file LIBPERM_TUNE_CACHE
// names when that is set.
// ---------------------------------------------------------------------------
namespace {

struct TuneChoice {
    PlanShape shape;
    float ms = 0.f;      // the batched candidate's time (0: nothing tuned)
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneChoice> g_tune;

bool tune_cache_lookup(int dev, int dtype, int n_max, TuneChoice* c) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, dtype, n_max));
    if (it != g_tune.end()) { *c = it->second; return true; }
    const char* path = getenv("LIBPERM_TUNE_CACHE");
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char name[256];
    int fd, fn, th, m, bn, lt, ms_, lg;
    float ms;
    bool found = false;
    while (fscanf(f, "%255s %d %d %d %d %d %d %d %d %f", name, &fd, &fn, &th, &m, &bn, &lt, &ms_, &lg, &ms) == 10) {
        if (strcmp(name, "perm-tune2") == 0 && fd == dtype && fn == n_max) {
            c->shape.threads = th;
            c->shape.m_low = m;
            c->shape.batch_nmax = bn;
            c->shape.layer_threads = lt;
            c->shape.m_single = ms_;
            c->shape.layer_grid_mult = lg;
            c->ms = ms;
            found = true;
        }
    }
    fclose(f);
    if (found) g_tune[std::make_tuple(dev, dtype, n_max)] = *c;
    return found;
}

void tune_cache_store(int dev, int dtype, int n_max, const TuneChoice& c) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[std::make_tuple(dev, dtype, n_max)] = c;
    if (const char* path = getenv("LIBPERM_TUNE_CACHE")) {
        if (FILE* f = fopen(path, "a")) {
            const PlanShape& s = c.shape;
            fprintf(f, "perm-tune2 %d %d %d %d %d %d %d %d %.4f\n", dtype, n_max, s.threads, s.m_low,
                    s.batch_nmax, s.layer_threads, s.m_single, s.layer_grid_mult, c.ms);
            fclose(f);
        }
    }
}

// Time one plan shape on `count` synthetic matrices of order n (device buffers given):
// the second of two calls, in milliseconds (-1 if the shape cannot run).
float time_shape(int n, perm_dtype dtype, const perm_opts& base, const PlanShape& shape, int n_max,
                 const void* d_mats, int count, void* d_out, cudaStream_t st) {
    perm_opts o = base;
    o.flags &= ~(PERM_FLAG_AUTOTUNE | PERM_FLAG_GRAPH | PERM_FLAG_PLAIN | PERM_FLAG_WIDE);
    o.max_batch = count;
    o.method = PERM_METHOD_SZ;
    perm_plan_t p = nullptr;
    if (plan_create_core(n_max, dtype, &o, nullptr, 0, shape, &p) != PERM_OK) return -1.f;
    std::vector<int> sizes(count, n);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = -1.f;
    bool ok = perm_batch(p, d_mats, sizes.data(), count, d_out, nullptr, st) == PERM_OK;   // warm-up
    if (ok) {
        cudaEventRecord(e0, st);
        ok = perm_batch(p, d_mats, sizes.data(), count, d_out, nullptr, st) == PERM_OK;
        cudaEventRecord(e1, st);
    }
    if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    perm_plan_destroy(p);
    cudaGetLastError();
    return ok ? ms : -1.f;
}

// Synthetic matrices for the tuner: a fixed LCG stream, complex entries of size
// about 1/n, or 0/1 entries.
std::vector<unsigned char> tune_matrices(perm_dtype dtype, int n, int count) {
    const size_t eb = dtype == PERM_C128 ? 16 : 8;
    std::vector<unsigned char> h((size_t)count * n * n * eb);
    unsigned long long x = 0x9E3779B97F4A7C15ull;
    for (size_t i = 0; i < (size_t)count * n * n; i++) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        if (dtype == PERM_C128) {
            double* d = reinterpret_cast<double*>(h.data()) + 2 * i;
            d[0] = ((double)(x >> 11) * 0x1.0p-53 - 0.5) / n;
            x = x * 6364136223846793005ull + 1442695040888963407ull;
            d[1] = ((double)(x >> 11) * 0x1.0p-53 - 0.5) / n;
        } else {
            reinterpret_cast<long long*>(h.data())[i] = (long long)((x >> 33) & 1ull);
        }
    }
    return h;
}

}  // namespace

static perm_status plan_create_tuned(int n_max, perm_dtype dtype, const perm_opts* opts,
                                     perm_plan_t* out) {
    perm_opts o = *opts;
    o.flags &= ~PERM_FLAG_AUTOTUNE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PERM_ECUDA;
    TuneChoice best;
    const bool uses_sz = o.method == PERM_METHOD_SZ || (o.method == PERM_METHOD_AUTO && auto_uses_sz(dtype));
    const int n0 = std::min(n_max, 20);      // the order the batched kernel is tuned at
    if (uses_sz && n0 >= 14 && !o.low_cols && !o.ctas_per_sm && !tune_cache_lookup(dev, dtype, n_max, &best)) {
        const int nbig = std::min(std::max(n_max, n0), 24);
        const int count = 2 * sms;
        std::vector<unsigned char> h = tune_matrices(dtype, nbig, count);
        void *dm = nullptr, *dout = nullptr;
        cudaStream_t st = nullptr;
        bool ok = cudaMalloc(&dm, h.size()) == cudaSuccess && cudaMalloc(&dout, (size_t)count * 32) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaMemcpy(dm, h.data(), h.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        // (1) batched kernel: CTA size x chain width (the matrices of order n0 are the first
        // n0 x n0 elements of each synthetic block, read as concatenated matrices)
        const int thr_c[3] = {256, 384, 512};
        const int thr_i[2] = {256, 512};
        const int* thr = dtype == PERM_C128 ? thr_c : thr_i;
        const int nthr = dtype == PERM_C128 ? 3 : 2;
        for (int ti = 0; ok && ti < nthr; ti++)
            for (int m = 11; m <= 13; m++) {
                PlanShape sh;
                sh.threads = thr[ti];
                sh.m_low = m;
                const float ms = time_shape(n0, dtype, o, sh, n0, dm, count, dout, st);
                if (ms > 0.f && (best.ms == 0.f || ms < best.ms)) { best.shape = sh; best.ms = ms; }
            }
        if (ok && best.ms > 0.f && dtype == PERM_C128 && n_max >= 21) {
            // (2) the batched / layer crossover, order by order while the batched kernel wins
            int cross = 18;
            for (int n = 19; n <= std::min(n_max, 22); n++) {
                PlanShape b = best.shape, l = best.shape;
                b.batch_nmax = 22;
                l.batch_nmax = 0;
                const float tb = time_shape(n, dtype, o, b, n, dm, count, dout, st);
                const float tl = time_shape(n, dtype, o, l, n, dm, count, dout, st);
                if (tb > 0.f && (tl <= 0.f || tb <= tl)) cross = n;
                else break;
            }
            best.shape.batch_nmax = cross;
            // (3) the layer path's shape for orders up to kLayerSmallN, on eight matrices of order
            // nbig (at most kFlowMaxCount matrices take the dataflow launch, whose chain width
            // follows the order and the count)
            const int cand[4][3] = {{384, 12, 2}, {384, 12, 4}, {512, 13, 1}, {512, 12, 2}};
            float lbest = 0.f;
            for (const auto& c : cand) {
                PlanShape sh = best.shape;
                sh.layer_threads = c[0];
                sh.m_single = c[1];
                sh.layer_grid_mult = c[2];
                const float ms = time_shape(nbig, dtype, o, sh, nbig, dm, 2 * kFlowMaxCount, dout, st);
                if (ms > 0.f && (lbest == 0.f || ms < lbest)) {
                    lbest = ms;
                    best.shape.layer_threads = c[0];
                    best.shape.m_single = c[1];
                    best.shape.layer_grid_mult = c[2];
                }
            }
        }
        if (st) cudaStreamDestroy(st);
        if (dm) cudaFree(dm);
        if (dout) cudaFree(dout);
        cudaGetLastError();
        if (best.ms > 0.f) tune_cache_store(dev, dtype, n_max, best);
    }
    perm_plan_t p = nullptr;
    perm_status s = plan_create_core(n_max, dtype, &o, nullptr, 0, best.ms > 0.f ? best.shape : PlanShape{}, &p);
    if (s != PERM_OK) return s;
    if (p) p->tuned = best.ms > 0.f;
    *out = p;
    return PERM_OK;
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput (measurement helper).
// ---------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(256) fp64_fma_kernel(double* sink, long long iters, double a, double b) {
    double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (long long i = 0; i < iters; i++) {
        x0 = __fma_rn(x0, a, b); x1 = __fma_rn(x1, a, b); x2 = __fma_rn(x2, a, b); x3 = __fma_rn(x3, a, b);
        x4 = __fma_rn(x4, a, b); x5 = __fma_rn(x5, a, b); x6 = __fma_rn(x6, a, b); x7 = __fma_rn(x7, a, b);
    }
    const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 1234.5678) sink[blockIdx.x] = s;   // keeps the chains alive; practically never true
}

}  // namespace

extern "C" perm_status perm_measure_fp64_peak(double ms_target, double* flops_per_s) {
    if (!flops_per_s || !(ms_target > 0)) return PERM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERM_ECUDA;
    const int blocks = sms * 8, threads = 256;
    double* sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(double)) != cudaSuccess) return PERM_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    long long iters = 1024;
    float ms = 0.f;
    cudaError_t err = cudaSuccess;
    for (int round = 0; round < 8; round++) {
        cudaEventRecord(e0);
        fp64_fma_kernel<<<blocks, threads>>>(sink, iters, 1.0000000001, 1e-12);
        cudaEventRecord(e1);
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms >= 0.5 * ms_target) break;
        iters = (long long)(iters * std::min(16.0, std::max(2.0, ms_target / std::max(ms, 1e-3f))));
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || ms <= 0.f) return PERM_ECUDA;
    *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
    return PERM_OK;
}
