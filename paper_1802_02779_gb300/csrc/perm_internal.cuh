// perm_internal.cuh -- definitions shared by the libperm translation units.
//
// Notation (Su & Zheng, arXiv:1802.02779, Section 4): rows and columns are
// 0-based; for a column set S with |S| = k,
//     T_k[S] = per(rows 0..k-1, columns S),
//     T_k[S] = sum_{j in S, ascending} a[k-1][j] * T_{k-1}[S \ {j}]      (property 4)
// with T_1[{j}] = a[0][j].  per(A) = T_n[{0..n-1}].
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/libperm.h"

namespace perm {

constexpr int kMaxN = 40;          // largest order any path accepts
constexpr int kMaxNSZ = 35;        // Store-zechin: chains of 2^13 need t = n - 13 <= kMaxHigh
constexpr int kMaxLow = 13;        // chain width m (low columns): 2^13 entries fit shared memory
constexpr int kMaxHigh = 22;       // high columns t = n - m (binomial tables hold C(x, y), x < 24)
// From this order on complex chain tables keep (Re, Im) of every entry only, 16 bytes instead of
// 24: the outer terms recompute w = Re + Im (one FP64 operation more per outer term, about 19 %
// more work at n = 34) and the tables take two thirds of the memory (n = 34: 92 GB instead of
// 139 GB; n = 35: 185 GB).  A function of n alone, so results do not depend on the path.
constexpr int kCompactN = 33;

// Low-column count actually used for an n x n matrix when `m_param` is requested.
__host__ __device__ inline int sz_low_for(int n, int m_param) {
    int m = m_param < n ? m_param : n;
    if (n - m > kMaxHigh) m = n - kMaxHigh;
    return m;
}

// One matrix of a batch.
struct ItemDesc {
    long long offset;   // first element of the matrix in `mats`
    int n;
    int out_index;      // slot in `out` / `item_status`
};

// ---------------------------------------------------------------------------
// double-double helpers (TwoSum: Knuth, TAOCP vol. 2, 4.2.2; TwoProduct via
// fma: Ogita, Rump & Oishi 2005).  Explicit _rn intrinsics so that nothing is
// contracted or reassociated.
// ---------------------------------------------------------------------------
struct dd2 { double hi, lo; };

__device__ __forceinline__ dd2 dd_two_sum(double a, double b) {
    double s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dd2 dd_fast_two_sum(double a, double b) {
    double s = __dadd_rn(a, b);
    double e = __dsub_rn(b, __dsub_rn(s, a));
    return {s, e};
}
// x + y for two double-doubles (accurate variant).
__device__ __forceinline__ dd2 dd_add(dd2 x, dd2 y) {
    dd2 s = dd_two_sum(x.hi, y.hi);
    dd2 t = dd_two_sum(x.lo, y.lo);
    double e = __dadd_rn(s.lo, t.hi);
    dd2 u = dd_fast_two_sum(s.hi, e);
    e = __dadd_rn(u.lo, t.lo);
    return dd_fast_two_sum(u.hi, e);
}
// x + a*b with the product taken exactly.
__device__ __forceinline__ dd2 dd_add_prod(dd2 x, double a, double b) {
    double p = __dmul_rn(a, b);
    double e = __fma_rn(a, b, -p);
    return dd_add(x, dd2{p, e});
}
__device__ __forceinline__ double dd_round(dd2 x) { return __dadd_rn(x.hi, x.lo); }

// ---------------------------------------------------------------------------
// Integer width decision (exactness of the modular arithmetic).
// Store-zechin and Ryser are polynomial identities over the integers, so
// evaluating them modulo 2^w yields per(A) mod 2^w, which equals per(A) when
// 0 <= per(A) < 2^w.  The width is the smallest of 64/128 (and 192 where the
// caller allows it) that an upper bound on per(A) allows.
// ---------------------------------------------------------------------------
enum : int { kWidth64 = 64, kWidth128 = 128, kWidth192 = 192, kWidthOverflow = 0, kWidthInvalid = -1 };

// Saturating 128-bit product (saturates at 2^128 - 1).
__device__ __forceinline__ unsigned __int128 sat_mul128(unsigned __int128 a, unsigned long long b) {
    if (a == 0 || b == 0) return 0;
    const unsigned __int128 maxv = ~(unsigned __int128)0;
    if (a > maxv / b) return maxv;
    return a * b;
}

// Decide the width for one integer matrix (row-major int64, n x n).  Checks
// the entries: negative -> invalid; for 0/1 input, anything else -> invalid.
// Bounds: per(A) <= prod_i r_i and <= prod_j c_j (row/column sums); for 0/1
// matrices also Bregman's bound per(A) <= prod_i (r_i!)^(1/r_i) (Bregman,
// Soviet Math. Dokl. 14 (1973)).  The 64- and 128-bit tests on the products
// are exact; the Bregman test and the 192-bit test compare log2 of the bound
// with a 0.01-bit margin (the rounding error of a sum of at most 80 log2
// terms is below 1e-12 bits).  Executed by one thread.
__device__ inline int decide_width(const long long* a, int n, bool zero_one, bool allow192 = false) {
    unsigned __int128 prow = 1, pcol = 1;
    double breg = 0.0, lrow = 0.0, lcol = 0.0;
    for (int i = 0; i < n; i++) {
        unsigned long long rs = 0;
        for (int j = 0; j < n; j++) {
            long long v = a[(size_t)i * n + j];
            if (v < 0 || (zero_one && v > 1)) return kWidthInvalid;
            if (v > (1ll << 40)) return kWidthInvalid;   // row sums must stay far below 2^63
            rs += (unsigned long long)v;
        }
        prow = sat_mul128(prow, rs);
        lrow += log2((double)rs);
        if (zero_one && rs > 1) {
            double lf = 0.0;
            for (unsigned long long q = 2; q <= rs; q++) lf += log2((double)q);
            breg += lf / (double)rs;
        }
    }
    for (int j = 0; j < n; j++) {
        unsigned long long cs = 0;
        for (int i = 0; i < n; i++) cs += (unsigned long long)a[(size_t)i * n + j];
        pcol = sat_mul128(pcol, cs);
        lcol += log2((double)cs);
    }
    unsigned __int128 b = prow < pcol ? prow : pcol;
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned __int128 maxv = ~(unsigned __int128)0;
    if (b < two64) return kWidth64;      // also every matrix with a zero row or column
    if (zero_one && breg < 63.99) return kWidth64;
    if (b < maxv) return kWidth128;
    if (zero_one && breg < 127.99) return kWidth128;
    if (allow192) {
        const double lb = lrow < lcol ? lrow : lcol;
        if (lb < 191.99 || (zero_one && breg < 191.99)) return kWidth192;
    }
    return kWidthOverflow;
}

// decide_width for one matrix by a whole warp (every lane calls it, with the
// same arguments).  Lanes compute the row and column terms; lane 0 combines
// them in the order decide_width uses, so every decision (and every rounding of
// the log2 sums) is identical to it.  The result is returned to every lane.
__device__ inline int decide_width_warp(const long long* a, int n, bool zero_one, bool allow192) {
    const int lane = threadIdx.x & 31;
    // row / column i = lane (slot 0) and i = lane + 32 (slot 1), kept in scalars
    unsigned long long rs0 = 0ull, rs1 = 0ull, cs0 = 0ull, cs1 = 0ull;
    double lr0 = 0.0, lr1 = 0.0, lc0 = 0.0, lc1 = 0.0, bt0 = 0.0, bt1 = 0.0;
    bool bad = false;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int i = lane + 32 * h;
        if (i < n) {
            unsigned long long rs = 0, cs = 0;
            for (int j = 0; j < n; j++) {
                const long long v = a[(size_t)i * n + j];
                if (v < 0 || (zero_one && v > 1) || v > (1ll << 40)) bad = true;
                rs += (unsigned long long)v;
                cs += (unsigned long long)a[(size_t)j * n + i];
            }
            double bt = 0.0;
            if (zero_one && rs > 1) {
                double lf = 0.0;
                for (unsigned long long q = 2; q <= rs; q++) lf += log2((double)q);
                bt = lf / (double)rs;
            }
            if (h == 0) { rs0 = rs; cs0 = cs; lr0 = log2((double)rs); lc0 = log2((double)cs); bt0 = bt; }
            else { rs1 = rs; cs1 = cs; lr1 = log2((double)rs); lc1 = log2((double)cs); bt1 = bt; }
        }
    }
    if (__any_sync(0xffffffffu, bad)) return kWidthInvalid;
    unsigned __int128 prow = 1, pcol = 1;
    double breg = 0.0, lrow = 0.0, lcol = 0.0;
    for (int i = 0; i < n; i++) {               // row (and column) order, as decide_width
        const int src = i & 31;
        const bool hi = i >= 32;
        const unsigned long long rs = __shfl_sync(0xffffffffu, hi ? rs1 : rs0, src);
        const unsigned long long cs = __shfl_sync(0xffffffffu, hi ? cs1 : cs0, src);
        const double lr = __shfl_sync(0xffffffffu, hi ? lr1 : lr0, src);
        const double lc = __shfl_sync(0xffffffffu, hi ? lc1 : lc0, src);
        const double bt = __shfl_sync(0xffffffffu, hi ? bt1 : bt0, src);
        prow = sat_mul128(prow, rs);
        pcol = sat_mul128(pcol, cs);
        lrow += lr;
        lcol += lc;
        if (zero_one && rs > 1) breg += bt;
    }
    const unsigned __int128 b = prow < pcol ? prow : pcol;
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned __int128 maxv = ~(unsigned __int128)0;
    if (b < two64) return kWidth64;
    if (zero_one && breg < 63.99) return kWidth64;
    if (b < maxv) return kWidth128;
    if (zero_one && breg < 127.99) return kWidth128;
    if (allow192) {
        const double lb = lrow < lcol ? lrow : lcol;
        if (lb < 191.99 || (zero_one && breg < 191.99)) return kWidth192;
    }
    return kWidthOverflow;
}

__device__ __forceinline__ int width_status(int w) {
    return w == kWidthInvalid ? PERM_EINVAL : (w == kWidthOverflow ? PERM_EOVERFLOW : PERM_OK);
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the kernel translation units).
// ---------------------------------------------------------------------------

// Store-zechin chain layout: columns 0..m-1 are "low", m..n-1 "high" (t = n-m).
// A chain is the set of all (H, L) with a fixed high subset H and every low
// subset L; it holds 2^m entries.  Workspace for the chains of one matrix:
// two layers of C(t, floor(t/2)) chains.
size_t sz_matrix_workspace_bytes(int dtype, int n, int m);
int sz_smem_bytes(int dtype, int n, int m);                // dynamic shared memory per CTA
int sz_batched_occupancy(int dtype, int n_max, int m, int threads);   // resident CTAs per SM
int sz_c128_threads_valid(int threads);
int sz_int_threads_valid(int threads);
cudaError_t sz_init_tables();                              // once per device (idempotent)

// Integer results are written as `out_words` 64-bit words per matrix (2: a
// 128-bit slot; 4: a 256-bit slot, the words above the computed width zero).
// Complex results are always one double2.

// Batched: one CTA per matrix, persistent over `count` items (dynamic order by
// an atomic counter at *counter, which must be zero at launch).
cudaError_t sz_launch_batched(int dtype, const void* mats, const ItemDesc* items, int count,
                              int n_max, int m, int threads, void* out, int out_words,
                              int* item_status, void* workspace, size_t ws_per_cta, int grid,
                              unsigned* counter, cudaStream_t st);

// One matrix, all CTAs on the chains of one layer at a time (t+1 launches).
cudaError_t sz_launch_single(int dtype, const void* mats, long long offset, int n, int m,
                             int out_index, void* out, int out_words, int* item_status,
                             void* workspace, int grid_cap, cudaStream_t st);
// The same for `count` matrices of one order n (device descriptors `items`), all
// in each layer launch; matrix c of the list uses the workspace slice
// [c * ws_bytes_per_item, (c + 1) * ws_bytes_per_item), ws_bytes_per_item >=
// sz_matrix_workspace_bytes(dtype, n, m).
// threads: CTA size of the complex layer kernel, 384 (two CTAs per SM), 512 (one; also for 0)
// or 768 (one); every choice gives the same bits.
//
// Default shape of the complex layer path by order and by the number of matrices of that order
// in one launch (measured on GB300; every shape gives the same bits).
// - Up to order 24 and more than kFlowMaxCount matrices: chains of 2^12 entries at two
//   384-thread CTAs per SM. More and smaller chains fill the narrow first and last layers (one
//   n = 24 matrix 2.08 ms against 2.56 ms with 2^13).
// - Up to order 24 and at most kFlowMaxCount matrices (the dataflow launch): chains of
//   2^w, w = floor((n - 1 + floor(log2 count)) / 2) clamped to 9..12. The critical path through
//   the t + 1 layers is then what binds, and shorter chains shorten it until their predecessor
//   loads dominate. This w was within 5 % of the best of 9..12 at n = 16..24 and 1, 2 or 4
//   matrices: one n = 20 matrix 0.35 ms (0.43 with 2^11), four n = 18 matrices 0.30 ms (0.43
//   with 2^12), one n = 24 matrix 1.83 ms with 2^11.
// - Above order 24: chains of 2^13 at one 768-thread CTA per SM. One outer column fewer means
//   fewer predecessor loads (n = 28 25.6 ms against 32.3 ms, n = 32 447 ms against 572 ms).
constexpr int kLayerSmallN = 24;
constexpr int kFlowMaxCount = 4;   // the dataflow launch takes at most this many matrices of an order
inline void sz_layer_default_shape(int n, int count, int* m, int* threads) {
    *threads = n > kLayerSmallN ? 768 : 384;
    if (n > kLayerSmallN) {
        *m = 13;
    } else if (count <= kFlowMaxCount) {
        int lg = 0;
        for (int c = count; c > 1; c >>= 1) lg++;
        const int w = (n - 1 + lg) / 2;
        *m = w < 9 ? 9 : (w > 12 ? 12 : w);
    } else {
        *m = 12;
    }
}
cudaError_t sz_launch_layers(int dtype, const void* mats, const ItemDesc* items, int count, int n, int m,
                             void* out, int out_words, int* item_status, void* workspace,
                             size_t ws_bytes_per_item, int grid_cap, cudaStream_t st, int threads = 0);

// The layer path of `count` complex matrices of order n <= kLayerSmallN as one
// persistent dataflow launch (sz_flow_c128): chains start when their
// predecessors are done instead of at layer boundaries; the same bits as
// sz_launch_layers.  Matrix c uses [c * ws_bytes_per_item, ...) of the
// workspace, ws_bytes_per_item >= sz_flow_workspace_bytes(n, m) (three layer
// regions and the chains' done flags); *counter is zeroed here.  An item whose
// wait gives up reports PERM_ETIMEDOUT in item_status.  The grid is persistent:
// three 256-thread CTAs per SM for chains of up to 2^11 entries, else two of 384
// threads, over num_sms SMs.
size_t sz_flow_workspace_bytes(int n, int m);
cudaError_t sz_launch_flow(const void* mats, const ItemDesc* items, int count, int n, int m, void* out,
                           int* item_status, void* workspace, size_t ws_bytes_per_item, unsigned* counter,
                           int num_sms, cudaStream_t st);

// Ryser: every matrix's codes are cut into ryser_parts(dtype, n) CTA-sized
// pieces (a function of n only).  One launch per distinct order n.  allow192:
// integer widths up to 192 bits (requires out_words = 4).  widths: 2 * count
// ints of scratch (integer types).
long long ryser_parts(int dtype, int n);
size_t ryser_partial_bytes(int dtype);                   // bytes of one piece's partial sum
cudaError_t ryser_launch_group(int dtype, int n, const void* mats, const ItemDesc* items, int count,
                               void* partials, int* widths, void* out, int out_words, bool allow192,
                               int* item_status, int grid, cudaStream_t st);

// One matrix split into several launches (or GPUs): pieces [begin, end) of its
// ryser_parts(dtype, n) pieces, partial sums to partials[0 .. end - begin);
// then the finishing kernel over all of its pieces' partial sums (in piece
// order), which gives the bits ryser_launch_group gives.  `item`: one device
// descriptor; widths: 2 ints of scratch (integer types).
cudaError_t ryser_launch_pieces(int dtype, int n, const void* mats, const ItemDesc* item, long long begin,
                                long long end, void* partials, int* widths, bool allow192, int grid,
                                cudaStream_t st);
cudaError_t ryser_finish_one(int dtype, int n, const ItemDesc* item, const void* partials, void* out,
                             int out_words, int* item_status, cudaStream_t st);

// Load now every kernel a plan of this element type may launch (Ryser: orders
// 1..n_max).  The runtime otherwise loads a kernel at its first launch, and
// that load can wait for all work running on the device -- which would stall a
// thread that feeds several streams (the server).
cudaError_t sz_preload(int dtype);
cudaError_t ryser_preload(int dtype, int n_max);

// n = 0 items: per = 1.
cudaError_t launch_trivial(int dtype, const ItemDesc* items, int count, void* out, int out_words,
                           int* item_status, cudaStream_t st);

// Method of PERM_METHOD_AUTO.  Measured on GB300 (batches of 1..4096 matrices,
// n = 2..30): for integer inputs Ryser's register-resident Gray-code walk is
// faster than the Store-zechin tables at every order (1.1x at n <= 12, about
// 2x at n = 13..22, 3-12x at n >= 23, where the tables no longer fit one CTA's
// slice and the one-matrix layer path runs), because integer Store-zechin does
// one addition per table read and waits on memory; for complex inputs
// Store-zechin is faster from n = 10 on (1.3-1.6x), and within 10% below.  So
// AUTO evaluates complex matrices with Store-zechin where the tables fit and
// integer matrices with Ryser.
inline bool auto_uses_sz(int dtype) { return dtype == PERM_C128; }


}  // namespace perm
