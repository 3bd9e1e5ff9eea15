// ryser_kernels.cu -- Ryser's inclusion-exclusion formula (Su & Zheng,
// arXiv:1802.02779, Section 3.3, Eqs. (2)-(4)), the memory-free fallback.
//
// Integers: Eq. (4),  per(A) = (-1)^n sum_{S subset cols} (-1)^{|S|} prod_i sum_{j in S} a_ij,
// over all 2^n subsets, modulo 2^64 or 2^128 (exact under the bound chosen by
// decide_width).  The subsets are visited in binary-reflected Gray-code order,
// so consecutive subsets differ in one column and each row sum is updated by
// one addition (the reuse Section 3.3 asks for).
//
// Complex: the same inclusion-exclusion with the half-size Gray code of Glynn
// (Glynn, European J. Combin. 31 (2010)):
//     per(A) = 2^{-(n-1)} sum_{d in {+-1}^n, d_0 = +1} (prod_k d_k) prod_i sum_j d_j a_ij,
// 2^{n-1} terms instead of 2^n (the paper is silent on this halving; the
// integer path cannot use it because 2^{-(n-1)} does not exist modulo 2^w).
//
// Work split.  The 2^G codes of one matrix are cut into `parts` CTA-sized
// pieces of 2^17 codes (one piece when there are fewer), each piece into 256
// contiguous thread ranges.  The grid has one CTA per piece, so CTAs retire
// every few milliseconds and work on higher-priority streams can take their
// place.  A thread computes its first row sums directly
// (no drift), then walks its range with one column update per step.  Thread
// sums are FP64 (complex) or modular; the CTA sums them in double-double in a
// fixed tree, and a second kernel sums the pieces of each matrix in a fixed
// order.  The split depends only on n, so results do not depend on the batch
// or the grid.
#include "perm_internal.cuh"

#include <algorithm>
#include <vector>

namespace perm {

namespace {

constexpr int kRyserThreads = 256;
constexpr int kLogCodesPerPart = 17;   // one CTA covers 2^17 codes, then retires

__host__ __device__ inline int log_codes(int dtype, int n) {
    return dtype == PERM_C128 ? n - 1 : n;
}
__host__ __device__ inline long long parts_for(int dtype, int n) {
    const int lg = log_codes(dtype, n);
    return lg > kLogCodesPerPart ? (1ll << (lg - kLogCodesPerPart)) : 1ll;
}

struct CPartial { double re_hi, re_lo, im_hi, im_lo; };
struct IPartial { unsigned long long lo, hi, status, width; };

// ---------------------------------------------------------------------------
// Complex (Glynn), compile-time order N.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kRyserThreads)
ryser_c128_kernel(const double2* __restrict__ mats, const ItemDesc* __restrict__ items,
                  long long total_parts, CPartial* __restrict__ partials) {
    __shared__ double2 s_col[N > 0 ? N : 1][N > 0 ? N : 1];   // s_col[j][i] = 2 * a_ij
    __shared__ double2 s_row0[N > 0 ? N : 1];                  // full row sums sum_j a_ij (d = +1)
    __shared__ dd2 s_re[kRyserThreads], s_im[kRyserThreads];
    constexpr int G = N - 1;                                    // log2 of the code count
    constexpr long long kParts = (G > kLogCodesPerPart) ? (1ll << (G - kLogCodesPerPart)) : 1ll;
    constexpr int kLogPart = (G > kLogCodesPerPart) ? kLogCodesPerPart : G;
    constexpr int kLogThr = kLogPart >= 8 ? 8 : kLogPart;       // threads actually used = 2^kLogThr
    constexpr int kLogLen = kLogPart - kLogThr;                 // codes per thread = 2^kLogLen

    for (long long task = blockIdx.x; task < total_parts; task += gridDim.x) {
        // every matrix of one launch has order N, hence kParts pieces
        const ItemDesc d = items[task / kParts];
        const long long part = task % kParts;
        const double2* a = mats + d.offset;
        __syncthreads();
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e % N;
            const double2 v = a[e];
            s_col[j][i] = make_double2(2.0 * v.x, 2.0 * v.y);
        }
        if (threadIdx.x < N) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < N; j++) {
                const double2 v = a[threadIdx.x * N + j];
                sr = __dadd_rn(sr, v.x);
                si = __dadd_rn(si, v.y);
            }
            s_row0[threadIdx.x] = make_double2(sr, si);
        }
        __syncthreads();

        double acc_re = 0.0, acc_im = 0.0;
        if (threadIdx.x < (1 << kLogThr)) {
            const unsigned long long g0 =
                ((unsigned long long)part << kLogPart) + ((unsigned long long)threadIdx.x << kLogLen);
            unsigned long long gr = g0 ^ (g0 >> 1);          // d_j = -1 iff bit (j-1) of gr is set
            double rr[N > 0 ? N : 1], ri[N > 0 ? N : 1];
            // direct row sums: start from d = all +1, subtract 2 a_ij for every -1
#pragma unroll
            for (int i = 0; i < N; i++) { rr[i] = s_row0[i].x; ri[i] = s_row0[i].y; }
            for (int j = 1; j < N; j++) {
                if ((gr >> (j - 1)) & 1ull) {
#pragma unroll
                    for (int i = 0; i < N; i++) {
                        rr[i] = __dsub_rn(rr[i], s_col[j][i].x);
                        ri[i] = __dsub_rn(ri[i], s_col[j][i].y);
                    }
                }
            }
            int neg = __popcll(gr) & 1;
            const unsigned long long len = 1ull << kLogLen;
            for (unsigned long long st = 0; st < len; st++) {
                if (st > 0) {
                    const int b = __ffsll((long long)st) - 1;   // same flip for the whole warp
                    gr ^= 1ull << b;
                    const double sg = ((gr >> b) & 1ull) ? -1.0 : 1.0;
                    const int j = b + 1;
#pragma unroll
                    for (int i = 0; i < N; i++) {
                        rr[i] = __fma_rn(sg, s_col[j][i].x, rr[i]);
                        ri[i] = __fma_rn(sg, s_col[j][i].y, ri[i]);
                    }
                    neg ^= 1;
                }
                double pr = rr[0], pi = ri[0];
#pragma unroll
                for (int i = 1; i < N; i++) {
                    const double t1 = __dmul_rn(pi, ri[i]);
                    const double t2 = __dmul_rn(pi, rr[i]);
                    const double nr = __fma_rn(pr, rr[i], -t1);
                    const double ni = __fma_rn(pr, ri[i], t2);
                    pr = nr;
                    pi = ni;
                }
                if (neg) { acc_re = __dsub_rn(acc_re, pr); acc_im = __dsub_rn(acc_im, pi); }
                else { acc_re = __dadd_rn(acc_re, pr); acc_im = __dadd_rn(acc_im, pi); }
            }
        }
        // fixed-order CTA reduction in double-double
        s_re[threadIdx.x] = dd2{acc_re, 0.0};
        s_im[threadIdx.x] = dd2{acc_im, 0.0};
        __syncthreads();
        for (int w = kRyserThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                s_re[threadIdx.x] = dd_add(s_re[threadIdx.x], s_re[threadIdx.x + w]);
                s_im[threadIdx.x] = dd_add(s_im[threadIdx.x], s_im[threadIdx.x + w]);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            CPartial p{s_re[0].hi, s_re[0].lo, s_im[0].hi, s_im[0].lo};
            partials[task] = p;
        }
    }
}

// ---------------------------------------------------------------------------
// Integers (Eq. 4) modulo 2^64 / 2^128, compile-time order N.
// ---------------------------------------------------------------------------
struct U128 { unsigned long long lo, hi; };

__device__ __forceinline__ U128 u128_add(U128 a, U128 b) {
    const unsigned long long lo = a.lo + b.lo;
    return {lo, a.hi + b.hi + (lo < a.lo ? 1ull : 0ull)};
}
__device__ __forceinline__ U128 u128_sub(U128 a, U128 b) {
    const unsigned long long lo = a.lo - b.lo;
    return {lo, a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull)};
}
__device__ __forceinline__ U128 u128_mul_u64(U128 a, unsigned long long b) {
    return {a.lo * b, __umul64hi(a.lo, b) + a.hi * b};
}

template <int N, bool W128>
__device__ __forceinline__ void ryser_int_range(const long long (*s_col)[N > 0 ? N : 1],
                                                unsigned long long g0, int log_len, U128& acc) {
    // row sums of gray(g0) directly
    unsigned long long gr = g0 ^ (g0 >> 1);
    long long r[N > 0 ? N : 1];
#pragma unroll
    for (int i = 0; i < N; i++) r[i] = 0;
    for (int j = 0; j < N; j++) {
        if ((gr >> j) & 1ull) {
#pragma unroll
            for (int i = 0; i < N; i++) r[i] += s_col[j][i];
        }
    }
    // sign (-1)^(n - |S|)
    int neg = (N - __popcll(gr)) & 1;
    const unsigned long long len = 1ull << log_len;
    U128 a = acc;
    for (unsigned long long st = 0; st < len; st++) {
        if (st > 0) {
            const int j = __ffsll((long long)st) - 1;
            gr ^= 1ull << j;
            if ((gr >> j) & 1ull) {
#pragma unroll
                for (int i = 0; i < N; i++) r[i] += s_col[j][i];
            } else {
#pragma unroll
                for (int i = 0; i < N; i++) r[i] -= s_col[j][i];
            }
            neg ^= 1;
        }
        if (W128) {
            U128 p = {(unsigned long long)r[0], 0ull};
#pragma unroll
            for (int i = 1; i < N; i++) p = u128_mul_u64(p, (unsigned long long)r[i]);
            a = neg ? u128_sub(a, p) : u128_add(a, p);
        } else {
            unsigned long long p = (unsigned long long)r[0];
#pragma unroll
            for (int i = 1; i < N; i++) p *= (unsigned long long)r[i];
            a.lo = neg ? a.lo - p : a.lo + p;
        }
    }
    acc = a;
}

template <int N>
__global__ void __launch_bounds__(kRyserThreads)
ryser_int_kernel(const long long* __restrict__ mats, const ItemDesc* __restrict__ items,
                 long long total_parts, const int* __restrict__ widths,
                 IPartial* __restrict__ partials) {
    __shared__ long long s_col[N > 0 ? N : 1][N > 0 ? N : 1];   // s_col[j][i] = a_ij
    __shared__ U128 s_acc[kRyserThreads];
    __shared__ int s_width;
    constexpr int G = N;
    constexpr long long kParts = (G > kLogCodesPerPart) ? (1ll << (G - kLogCodesPerPart)) : 1ll;
    constexpr int kLogPart = (G > kLogCodesPerPart) ? kLogCodesPerPart : G;
    constexpr int kLogThr = kLogPart >= 8 ? 8 : kLogPart;
    constexpr int kLogLen = kLogPart - kLogThr;

    for (long long task = blockIdx.x; task < total_parts; task += gridDim.x) {
        const ItemDesc d = items[task / kParts];
        const long long part = task % kParts;
        const long long* a = mats + d.offset;
        __syncthreads();
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e % N;
            s_col[j][i] = a[e];
        }
        if (threadIdx.x == 0) s_width = widths[task / kParts];
        __syncthreads();
        const int w = s_width;
        U128 acc = {0ull, 0ull};
        if (threadIdx.x < (1 << kLogThr)) {
            const unsigned long long g0 =
                ((unsigned long long)part << kLogPart) + ((unsigned long long)threadIdx.x << kLogLen);
            if (w == kWidth64) ryser_int_range<N, false>(s_col, g0, kLogLen, acc);
            else ryser_int_range<N, true>(s_col, g0, kLogLen, acc);
        }
        s_acc[threadIdx.x] = acc;
        __syncthreads();
        for (int h = kRyserThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) s_acc[threadIdx.x] = u128_add(s_acc[threadIdx.x], s_acc[threadIdx.x + h]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            IPartial p;
            p.lo = s_acc[0].lo;
            p.hi = (w == kWidth64) ? 0ull : s_acc[0].hi;
            p.status = (unsigned long long)width_status(w);
            p.width = (unsigned long long)w;
            partials[task] = p;
        }
    }
}

// Sum the pieces of every matrix (fixed order) and write the results.
__global__ void ryser_finish_c128(const ItemDesc* items, long long parts, int count,
                                  const CPartial* partials, double2* out, int* item_status) {
    const int it = blockIdx.x;
    if (it >= count) return;
    __shared__ dd2 s_re[32], s_im[32];
    const long long b = (long long)it * parts, e = b + parts;
    dd2 re = {0.0, 0.0}, im = {0.0, 0.0};
    for (long long p = b + threadIdx.x; p < e; p += 32) {
        re = dd_add(re, dd2{partials[p].re_hi, partials[p].re_lo});
        im = dd_add(im, dd2{partials[p].im_hi, partials[p].im_lo});
    }
    s_re[threadIdx.x] = re;
    s_im[threadIdx.x] = im;
    __syncwarp();
    for (int w = 16; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s_re[threadIdx.x] = dd_add(s_re[threadIdx.x], s_re[threadIdx.x + w]);
            s_im[threadIdx.x] = dd_add(s_im[threadIdx.x], s_im[threadIdx.x + w]);
        }
        __syncwarp();
    }
    if (threadIdx.x == 0) {
        const int n = items[it].n;
        const double sc = ldexp(1.0, -(n - 1));     // exact power of two
        const double r = dd_round(dd2{s_re[0].hi * sc, s_re[0].lo * sc});
        const double i = dd_round(dd2{s_im[0].hi * sc, s_im[0].lo * sc});
        out[items[it].out_index] = make_double2(r, i);
        if (item_status) item_status[items[it].out_index] = PERM_OK;
    }
}

__global__ void ryser_finish_int(const ItemDesc* items, long long parts, int count,
                                 const IPartial* partials, unsigned long long* out,
                                 int* item_status) {
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= count) return;
    U128 s = {0ull, 0ull};
    int st = PERM_OK;
    bool w64 = false;
    for (long long p = (long long)it * parts; p < (long long)(it + 1) * parts; p++) {
        s = u128_add(s, U128{partials[p].lo, partials[p].hi});
        if (partials[p].status != PERM_OK) st = (int)partials[p].status;
        w64 = partials[p].width == (unsigned long long)kWidth64;
    }
    if (w64) s.hi = 0ull;       // the sum is only meaningful modulo 2^64
    const int o = items[it].out_index;
    out[2 * o] = s.lo;
    out[2 * o + 1] = s.hi;
    if (item_status) item_status[o] = st;
}

// Integer width of every matrix of a launch, once (one thread per matrix).
__global__ void ryser_widths_kernel(const long long* mats, const ItemDesc* items, int count, int n,
                                    int zero_one, int* widths) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) widths[i] = decide_width(mats + items[i].offset, n, zero_one != 0);
}

template <int N>
cudaError_t launch_n(int dtype, const void* mats, const ItemDesc* items, long long total_parts,
                     const int* widths, void* partials, int grid, cudaStream_t st) {
    const int g = (int)std::min<long long>(total_parts, (long long)grid);
    if (dtype == PERM_C128) {
        ryser_c128_kernel<N><<<g, kRyserThreads, 0, st>>>((const double2*)mats, items, total_parts,
                                                          (CPartial*)partials);
    } else {
        ryser_int_kernel<N><<<g, kRyserThreads, 0, st>>>((const long long*)mats, items, total_parts,
                                                         widths, (IPartial*)partials);
    }
    return cudaGetLastError();
}

typedef cudaError_t (*launch_fn)(int, const void*, const ItemDesc*, long long, const int*, void*, int,
                                 cudaStream_t);

template <int... Ns>
struct Table {
    static constexpr launch_fn fns[sizeof...(Ns)] = {&launch_n<Ns>...};
};

#define PERM_NS 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, \
                24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40
using NTable = Table<PERM_NS>;

}  // namespace


// Launch Ryser for `count` matrices that all have order n (1 <= n <= 40);
// `partials` holds count * ryser_parts(dtype, n) 32-byte slots and `widths`
// count ints (integer types only).
cudaError_t ryser_launch_group(int dtype, int n, const void* mats, const ItemDesc* items, int count,
                               void* partials, int* widths, void* out, int* item_status, int grid,
                               cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (n < 1 || n > kMaxN) return cudaErrorInvalidValue;
    const long long parts = parts_for(dtype, n);
    if (dtype != PERM_C128) {
        ryser_widths_kernel<<<(count + 127) / 128, 128, 0, st>>>((const long long*)mats, items, count, n,
                                                                 dtype == PERM_U01, widths);
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = NTable::fns[n - 1](dtype, mats, items, (long long)count * parts, widths, partials,
                                       grid, st);
    if (e != cudaSuccess) return e;
    if (dtype == PERM_C128)
        ryser_finish_c128<<<count, 32, 0, st>>>(items, parts, count, (const CPartial*)partials,
                                                (double2*)out, item_status);
    else
        ryser_finish_int<<<(count + 127) / 128, 128, 0, st>>>(items, parts, count,
                                                              (const IPartial*)partials,
                                                              (unsigned long long*)out, item_status);
    return cudaGetLastError();
}

long long ryser_parts(int dtype, int n) { return parts_for(dtype, n); }

}  // namespace perm
