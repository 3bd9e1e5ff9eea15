// ryser_kernels.cu -- Ryser's inclusion-exclusion formula (Su & Zheng,
// arXiv:1802.02779, Section 3.3, Eqs. (2)-(4)), the memory-free fallback.
//
// Integers: Eq. (4),  per(A) = (-1)^n sum_{S subset cols} (-1)^{|S|} prod_i sum_{j in S} a_ij,
// over all 2^n subsets, modulo 2^64, 2^128 or 2^192 (exact under the bound
// chosen by decide_width).  The subsets are visited in binary-reflected Gray-code order,
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
// pieces of 2^17 codes (2^16 for complex input; one piece when there are
// fewer), each piece into 256
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
#include <type_traits>
#include <vector>

namespace perm {

namespace {

constexpr int kRyserThreads = 256;
// One CTA covers 2^17 integer codes (2^16 for complex input, whose codes cost
// about 6n FP64 operations each: a CTA then runs ~3.5 ms at n = 34), then
// retires, so work on a higher-priority stream waits at most that long for SMs.
constexpr int kLogCodesPerPart = 17;
constexpr int kLogCodesPerPartC = 16;

__host__ __device__ inline int log_codes(int dtype, int n) {
    return dtype == PERM_C128 ? n - 1 : n;
}
__host__ __device__ inline long long parts_for(int dtype, int n) {
    const int lg = log_codes(dtype, n);
    const int per = dtype == PERM_C128 ? kLogCodesPerPartC : kLogCodesPerPart;
    return lg > per ? (1ll << (lg - per)) : 1ll;
}

struct CPartial { double re_hi, re_lo, im_hi, im_lo; };
// meta: item status in bits 0..31, the width computed (0, 64, 128, 192) in bits
// 32..47, and the right shift the finished sum needs (n - 1 for Glynn's form,
// else 0) in bits 48..55
struct IPartial { unsigned long long w[4], meta; };

// ---------------------------------------------------------------------------
// Complex (Glynn), compile-time order N.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kRyserThreads)
ryser_c128_kernel(const double2* __restrict__ mats, const ItemDesc* __restrict__ items,
                  long long total_parts, long long part0, long long item_parts,
                  CPartial* __restrict__ partials) {
    __shared__ double2 s_col[N > 0 ? N : 1][N > 0 ? N : 1];   // s_col[j][i] = 2 * a_ij
    __shared__ double2 s_row0[N > 0 ? N : 1];                  // full row sums sum_j a_ij (d = +1)
    __shared__ dd2 s_re[kRyserThreads], s_im[kRyserThreads];
    constexpr int G = N - 1;                                    // log2 of the code count
    constexpr long long kParts = (G > kLogCodesPerPartC) ? (1ll << (G - kLogCodesPerPartC)) : 1ll;
    constexpr int kLogPart = (G > kLogCodesPerPartC) ? kLogCodesPerPartC : G;
    constexpr int kLogThr = kLogPart >= 8 ? 8 : kLogPart;       // threads actually used = 2^kLogThr
    constexpr int kLogLen = kLogPart - kLogThr;                 // codes per thread = 2^kLogLen

    for (long long task = blockIdx.x; task < total_parts; task += gridDim.x) {
        // every matrix of one launch has order N, hence kParts pieces; a launch takes
        // pieces part0 .. part0 + item_parts - 1 of each (all of them unless a caller
        // splits one matrix's pieces over several launches or GPUs)
        const ItemDesc d = items[task / item_parts];
        const long long part = part0 + task % item_parts;
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
// Integers (Eq. 4) modulo 2^64, 2^128 or 2^192, compile-time order N.
//
// Row sums r_i(S) = sum_{j in S} a_ij are updated by one column per Gray step.
// 0/1 input (ZO): r_i <= N <= 40, so the row sums are 32-bit and six of them
// multiply exactly in 32 bits (40^6 < 2^32); the running product then takes
// one 32-bit factor per group of six rows, limb by limb.  Other integers:
// 64-bit row sums and factors, with two independent product chains (even and
// odd rows) for instruction-level parallelism.  Every grouping is the same
// product modulo 2^W, so results do not depend on it.
// ---------------------------------------------------------------------------
struct U128 { unsigned long long lo, hi; };

__device__ __forceinline__ U128 u128_mul_u64(U128 a, unsigned long long b) {
    return {a.lo * b, __umul64hi(a.lo, b) + a.hi * b};
}
__device__ __forceinline__ U128 u128_mul(U128 a, U128 b) {
    return {a.lo * b.lo, __umul64hi(a.lo, b.lo) + a.lo * b.hi + a.hi * b.lo};
}

// Integer accumulators: up to four 64-bit words (Glynn's sum modulo 2^(192+n-1)
// needs four at n >= 34).
constexpr int kAccWords = 4;
typedef unsigned long long AccWords[kAccWords];

// acc += x / acc -= x over the low K words (K = 1..4), carries propagated.
template <int K, int NA, int NX>
__device__ __forceinline__ void words_add(unsigned long long (&acc)[NA], const unsigned long long (&x)[NX]) {
    static_assert(K <= NA && K <= NX, "word count");
    if constexpr (K == 1) {
        acc[0] += x[0];
    } else if constexpr (K == 2) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;"
            : "+l"(acc[0]), "+l"(acc[1]) : "l"(x[0]), "l"(x[1]));
    } else if constexpr (K == 3) {
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
            : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]) : "l"(x[0]), "l"(x[1]), "l"(x[2]));
    } else {
        asm("add.cc.u64 %0, %0, %4;\n\taddc.cc.u64 %1, %1, %5;\n\taddc.cc.u64 %2, %2, %6;\n\t"
            "addc.u64 %3, %3, %7;"
            : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]), "+l"(acc[3])
            : "l"(x[0]), "l"(x[1]), "l"(x[2]), "l"(x[3]));
    }
}
template <int K, int NA, int NX>
__device__ __forceinline__ void words_sub(unsigned long long (&acc)[NA], const unsigned long long (&x)[NX]) {
    static_assert(K <= NA && K <= NX, "word count");
    if constexpr (K == 1) {
        acc[0] -= x[0];
    } else if constexpr (K == 2) {
        asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;"
            : "+l"(acc[0]), "+l"(acc[1]) : "l"(x[0]), "l"(x[1]));
    } else {
        asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
            : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]) : "l"(x[0]), "l"(x[1]), "l"(x[2]));
    }
}

// p *= g modulo 2^(32 L), p in 32-bit limbs (least significant first).
template <int L>
__device__ __forceinline__ void limbs_mul_u32(unsigned (&p)[L], unsigned g) {
    unsigned carry = 0;
#pragma unroll
    for (int k = 0; k < L - 1; k++) {
        const unsigned long long t = (unsigned long long)p[k] * g + carry;   // < 2^64
        p[k] = (unsigned)t;
        carry = (unsigned)(t >> 32);
    }
    p[L - 1] = p[L - 1] * g + carry;
}

// prod_i r_i modulo 2^W into x[0..W/64-1].
template <int N, int W>
__device__ __forceinline__ void row_product(const unsigned (&r)[N], AccWords& x) {
    constexpr int kGroups = (N + 5) / 6;
    unsigned g[kGroups];
#pragma unroll
    for (int q = 0; q < kGroups; q++) {
        g[q] = r[6 * q];
#pragma unroll
        for (int i = 6 * q + 1; i < 6 * q + 6 && i < N; i++) g[q] *= r[i];
    }
    if constexpr (W == 64) {
        unsigned long long p = g[0];
#pragma unroll
        for (int q = 1; q < kGroups; q++) p *= (unsigned long long)g[q];
        x[0] = p;
    } else {
        constexpr int L = W / 32;
        unsigned p[L];
        p[0] = g[0];
#pragma unroll
        for (int k = 1; k < L; k++) p[k] = 0u;
#pragma unroll
        for (int q = 1; q < kGroups; q++) limbs_mul_u32<L>(p, g[q]);
#pragma unroll
        for (int k = 0; k < W / 64; k++) x[k] = (unsigned long long)p[2 * k] | ((unsigned long long)p[2 * k + 1] << 32);
    }
}
template <int N, int W>
__device__ __forceinline__ void row_product(const unsigned long long (&r)[N], AccWords& x) {
    if constexpr (N == 1) {
        x[0] = r[0];
        if constexpr (W >= 128) x[1] = 0ull;
        if constexpr (W >= 192) x[2] = 0ull;
    } else if constexpr (W == 64) {
        unsigned long long pa = r[0], pb = r[1];
#pragma unroll
        for (int i = 2; i < N; i++) {
            if (i & 1) pb *= r[i];
            else pa *= r[i];
        }
        x[0] = pa * pb;
    } else if constexpr (W == 128) {
        U128 pa = {r[0], 0ull}, pb = {r[1], 0ull};
#pragma unroll
        for (int i = 2; i < N; i++) {
            if (i & 1) pb = u128_mul_u64(pb, r[i]);
            else pa = u128_mul_u64(pa, r[i]);
        }
        const U128 p = u128_mul(pa, pb);
        x[0] = p.lo;
        x[1] = p.hi;
    } else {
        unsigned long long w0 = r[0], w1 = 0ull, w2 = 0ull;
#pragma unroll
        for (int i = 1; i < N; i++) {
            const unsigned long long b = r[i];
            const unsigned long long h0 = __umul64hi(w0, b), h1 = __umul64hi(w1, b);
            const unsigned long long t1 = w1 * b;
            const unsigned long long n1 = t1 + h0;
            w2 = w2 * b + h1 + (n1 < t1 ? 1ull : 0ull);
            w1 = n1;
            w0 = w0 * b;
        }
        x[0] = w0;
        x[1] = w1;
        x[2] = w2;
    }
}

// One thread's contiguous range of 2^log_len Gray codes starting at code g0.
// s_col: column j of A at s_col[j * NP .. j * NP + N - 1].
template <int N, int NP, int W, typename E>
__device__ __forceinline__ void ryser_int_range(const E* __restrict__ s_col, unsigned long long g0,
                                                int log_len, AccWords& acc) {
    constexpr int K = W / 64;
    const unsigned long long gr0 = g0 ^ (g0 >> 1);
    E r[N];
#pragma unroll
    for (int i = 0; i < N; i++) r[i] = 0;
    for (int j = 0; j < N; j++) {
        if ((gr0 >> j) & 1ull) {
#pragma unroll
            for (int i = 0; i < N; i++) r[i] += s_col[j * NP + i];
        }
    }
    // sign (-1)^(n - |S|)
    int neg = (N - __popcll(gr0)) & 1;
    // log_len <= 9 and g0 is a multiple of 2^log_len: the walk flips only low bits
    unsigned grl = (unsigned)gr0;
    const unsigned len = 1u << log_len;
    unsigned long long a[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = acc[k];
    for (unsigned st = 0; st < len; st++) {
        if (st > 0) {
            const int j = __ffs(st) - 1;                // the same column for the whole warp
            grl ^= 1u << j;
            const E* col = s_col + j * NP;
            if ((grl >> j) & 1u) {
#pragma unroll
                for (int i = 0; i < N; i++) r[i] += col[i];
            } else {
#pragma unroll
                for (int i = 0; i < N; i++) r[i] -= col[i];
            }
            neg ^= 1;
        }
        AccWords x;
        row_product<N, W>(r, x);
        if (neg) words_sub<K>(a, x);
        else words_add<K>(a, x);
    }
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = a[k];
}

// ---------------------------------------------------------------------------
// 0/1 matrices by Glynn's formula, exactly.  With d_0 = +1 and d_1..d_{n-1} in
// {+1, -1},
//     Sum_d (prod_k d_k) prod_i rho_i(d) = 2^{n-1} per(A),   rho_i(d) = sum_j d_j a_ij,
// an identity over the integers (each permutation's term survives with
// coefficient 2^{n-1}; every other monomial cancels).  The sum is therefore a
// multiple of 2^{n-1}: computed modulo 2^{w+n-1} and shifted right by n-1 it
// gives per(A) modulo 2^w exactly, over 2^{n-1} codes instead of Eq. (4)'s 2^n.
// |rho_i| <= R_i (the row sum), so when every R_i <= B a group of G rows with
// B^G < 2^31 multiplies exactly in signed 32 bits (B = n for 0/1 input; for
// other integers B = 127 or 32767, chosen per matrix); the group magnitudes
// multiply limb by limb modulo 2^{32 L}, L = ceil((w + n - 1) / 32), and the
// sign is applied when accumulating.
// ---------------------------------------------------------------------------
template <unsigned long long B, int N>
constexpr int glynn_group() {
    int g = 1;
    unsigned long long p = B;
    while (g < N && p * B < (1ull << 31)) {
        p *= B;
        g++;
    }
    return g;
}
constexpr unsigned long long kRowBound1 = 127, kRowBound2 = 32767;   // integer row-sum classes 1, 2

// One thread's range of 2^log_len Glynn codes starting at g0: d_j = -1 iff bit
// j - 1 of gray(code) is set.  s_col2[j * NP + i] = 2 a_ij, s_row[i] = sum_j a_ij.
// log_len <= 8, and g0 is a multiple of 2^log_len, so the walk flips only the
// low 8 bits of the Gray code (32-bit counters).
//
// For 0/1 input many terms vanish: rho_i is a sum of +-1 over the ones of row
// i, zero for about a fifth of the sign vectors when R_i is even, so at density
// 1/2 and n = 20 about 88% of the products are zero.  A zero group product
// skips the wide product and the accumulation (a branch taken by a whole warp
// only when every lane's term vanishes).  A negative term is added as the
// complement of its magnitude, and the +1 each complement lacks is added once
// at the end from a count.  G: rows per exact 32-bit group.
template <int N, int NP, int L, int G>
__device__ __forceinline__ void glynn_range(const int* __restrict__ s_col2, const int* __restrict__ s_row,
                                            unsigned long long g0, int log_len,
                                            AccWords& acc) {
    constexpr int K = (L + 1) / 2;                 // 64-bit words of the accumulator
    constexpr int kGroups = (N + G - 1) / G;
    const unsigned long long gr0 = g0 ^ (g0 >> 1);
    int r[N];
#pragma unroll
    for (int i = 0; i < N; i++) r[i] = s_row[i];
    for (int j = 1; j < N; j++) {
        if ((gr0 >> (j - 1)) & 1ull) {
#pragma unroll
            for (int i = 0; i < N; i++) r[i] -= s_col2[j * NP + i];
        }
    }
    unsigned neg = (unsigned)__popcll(gr0) & 1u;   // prod_k d_k = (-1)^neg
    unsigned grl = (unsigned)gr0;                   // low word of the Gray code
    unsigned ncount = 0;                            // negative terms added as complements
    const unsigned len = 1u << log_len;
    unsigned long long a[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = acc[k];
    for (unsigned st = 0; st < len; st++) {
        if (st > 0) {
            const int b = __ffs(st) - 1;            // the same flip for the whole warp
            grl ^= 1u << b;
            const int* col = s_col2 + (b + 1) * NP;
            if ((grl >> b) & 1u) {
#pragma unroll
                for (int i = 0; i < N; i++) r[i] -= col[i];
            } else {
#pragma unroll
                for (int i = 0; i < N; i++) r[i] += col[i];
            }
            neg ^= 1u;
        }
        int g[kGroups];
        bool nonzero = true;
#pragma unroll
        for (int q = 0; q < kGroups; q++) {
            g[q] = r[q * G];
#pragma unroll
            for (int i = q * G + 1; i < q * G + G && i < N; i++) g[q] *= r[i];
            nonzero = nonzero && g[q] != 0;
        }
        if (nonzero) {
            unsigned sgn = neg;
            unsigned p[L];
#pragma unroll
            for (int q = 0; q < kGroups; q++) sgn ^= (unsigned)g[q] >> 31;
            p[0] = (unsigned)abs(g[0]);
#pragma unroll
            for (int k = 1; k < L; k++) p[k] = 0u;
#pragma unroll
            for (int q = 1; q < kGroups; q++) limbs_mul_u32<L>(p, (unsigned)abs(g[q]));
            // sgn ? ~|P| : |P| modulo 2^(64 K); the missing +1 of -|P| = ~|P| + 1 is counted
            const unsigned long long m = 0ull - (unsigned long long)sgn;
            unsigned long long x[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                const unsigned long long hi = (2 * k + 1 < L) ? ((unsigned long long)p[2 * k + 1] << 32) : 0ull;
                x[k] = ((unsigned long long)p[2 * k] | hi) ^ m;
            }
            words_add<K>(a, x);
            ncount += sgn;
        }
    }
    unsigned long long c[K];
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = k == 0 ? (unsigned long long)ncount : 0ull;
    words_add<K>(a, c);
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = a[k];
}

// Bit-sliced variant for 12 <= n <= 40 (full warps, one word per row set).
// Let c_i be the number of ones of row i among the columns with d_j = -1, so that
// rho_i = R_i - 2 c_i.  A thread keeps the c_i of all rows as bit planes
// (plane k holds bit k of every c_i): flipping column j adds or subtracts the
// column's row mask with a ripple over the planes, and "some rho_i = 0" is the
// plane-wise test c_i == R_i / 2 over the rows of even R_i -- a few logical
// operations per code for every row at once.  The codes whose product is
// nonzero (about 6% at density 1/2, n = 20) go into a per-warp queue; every 32
// queued codes are evaluated by the whole warp from scratch (rho_i by popcount of
// the code against row i's ones), so the rare wide products keep all lanes busy.
template <int N>
constexpr int count_planes() {
    int p = 1;
    while ((1 << p) <= N) p++;
    return p;                     // bits of 0..N
}

__device__ __forceinline__ int popcnt(unsigned x) { return __popc(x); }
__device__ __forceinline__ int popcnt(unsigned long long x) { return __popcll(x); }

// The Glynn term of one code (d_j = -1 iff bit j - 1 of `code`), added to `a` as
// described for glynn_range.  s_rm[i]: bit j - 1 set iff a_ij = 1 (j >= 1).
// M: an unsigned type wide enough for n rows (32 or 64 bits).
template <int N, int L, typename M>
__device__ __forceinline__ void glynn_term_from_code(M code, const M* __restrict__ s_rm,
                                                     const int* __restrict__ s_row,
                                                     unsigned long long (&a)[(L + 1) / 2], unsigned& ncount) {
    constexpr int K = (L + 1) / 2;
    constexpr int G = glynn_group<N, N>();
    constexpr int kGroups = (N + G - 1) / G;
    unsigned sgn = (unsigned)popcnt(code) & 1u;
    int g[kGroups];
#pragma unroll
    for (int q = 0; q < kGroups; q++) {
        g[q] = s_row[q * G] - 2 * popcnt(code & s_rm[q * G]);
#pragma unroll
        for (int i = q * G + 1; i < q * G + G && i < N; i++) g[q] *= s_row[i] - 2 * popcnt(code & s_rm[i]);
        sgn ^= (unsigned)g[q] >> 31;
    }
    unsigned p[L];
    p[0] = (unsigned)abs(g[0]);
#pragma unroll
    for (int k = 1; k < L; k++) p[k] = 0u;
#pragma unroll
    for (int q = 1; q < kGroups; q++) limbs_mul_u32<L>(p, (unsigned)abs(g[q]));
    const unsigned long long m = 0ull - (unsigned long long)sgn;
    unsigned long long x[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        const unsigned long long hi = (2 * k + 1 < L) ? ((unsigned long long)p[2 * k + 1] << 32) : 0ull;
        x[k] = ((unsigned long long)p[2 * k] | hi) ^ m;
    }
    words_add<K>(a, x);
    ncount += sgn;
}

// One thread's range of 2^log_len codes from g0 (a multiple of 2^log_len);
// called by every lane of full warps with the same log_len.  q: this warp's
// 64-entry queue.  s_cm[j]: bit i set iff a_ij = 1.  M: row-set words (32 bits
// for n <= 32, else 64).
template <int N, int L, typename M>
__device__ __forceinline__ void glynn_bits_range(const M* __restrict__ s_cm, const M* __restrict__ s_rm,
                                                 const int* __restrict__ s_row, M* q,
                                                 M g0, int log_len, AccWords& acc) {
    constexpr int K = (L + 1) / 2;
    constexpr int NPL = count_planes<N>();
    const unsigned lane = threadIdx.x & 31u;
    M gr = g0 ^ (g0 >> 1);
    // target planes: rows of even R_i, h_i = R_i / 2
    M H[NPL], P[NPL];
    M even = 0;
#pragma unroll
    for (int k = 0; k < NPL; k++) { H[k] = 0; P[k] = 0; }
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int R = s_row[i];
        const unsigned c = (unsigned)popcnt(gr & s_rm[i]);
        if ((R & 1) == 0) even |= (M)1 << i;
#pragma unroll
        for (int k = 0; k < NPL; k++) {
            H[k] |= (M)(((unsigned)(R >> 1) >> k) & 1u) << i;
            P[k] |= (M)((c >> k) & 1u) << i;
        }
    }
    unsigned qn = 0;                 // entries in the queue (the same in every lane)
    unsigned ncount = 0;
    unsigned long long a[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = acc[k];
    const unsigned len = 1u << log_len;
    for (unsigned st = 0; st < len; st++) {
        if (st > 0) {
            const int b = __ffs(st) - 1;     // the same flip for the whole warp
            gr ^= (M)1 << b;
            const M msk = s_cm[b + 1];
            if ((gr >> b) & 1u) {            // d_{b+1}: +1 -> -1, c_i += 1 on the rows of msk
                M cy = msk;
#pragma unroll
                for (int k = 0; k < NPL; k++) { const M t = P[k] & cy; P[k] ^= cy; cy = t; }
            } else {                         // -1 -> +1, c_i -= 1
                M bw = msk;
#pragma unroll
                for (int k = 0; k < NPL; k++) { const M t = ~P[k] & bw; P[k] ^= bw; bw = t; }
            }
        }
        M diff = 0;
#pragma unroll
        for (int k = 0; k < NPL; k++) diff |= P[k] ^ H[k];
        const bool live = (even & ~diff) == 0;    // no rho_i is zero
        const unsigned ball = __ballot_sync(0xffffffffu, live);
        if (ball) {
            if (live) q[qn + __popc(ball & ((1u << lane) - 1u))] = gr;
            qn += (unsigned)__popc(ball);
            if (qn >= 32u) {
                __syncwarp();
                const M code = q[lane];
                const M rest = lane < qn - 32u ? q[32u + lane] : (M)0;
                __syncwarp();
                if (lane < qn - 32u) q[lane] = rest;
                qn -= 32u;
                __syncwarp();
                glynn_term_from_code<N, L, M>(code, s_rm, s_row, a, ncount);
            }
        }
    }
    __syncwarp();
    if (lane < qn) glynn_term_from_code<N, L, M>(q[lane], s_rm, s_row, a, ncount);
    __syncwarp();
    unsigned long long c[K];
#pragma unroll
    for (int k = 0; k < K; k++) c[k] = k == 0 ? (unsigned long long)ncount : 0ull;
    words_add<K>(a, c);
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = a[k];
}

// Widest modulus an order-N matrix of the given kind can need: a 0/1 matrix
// has per(A) <= n!, and 20! < 2^64, 34! < 2^128, 40! < 2^192.
template <int N, bool ZO>
constexpr int max_width() {
    return !ZO ? 192 : (N <= 20 ? 64 : (N <= 34 ? 128 : 192));
}

// PATH (general integers only; 0/1 matrices use kPathAll): kPathGlynn takes
// the items with small row sums and a 64- or 128-bit width, kPathEq4 every
// other item; the two are launched one after the other over the same pieces,
// each writing only its own items' partial sums, so that each variant gets the
// registers of its own arithmetic.
enum : int { kPathAll = 0, kPathGlynn = 1, kPathEq4 = 2 };

template <int N, bool ZO, int PATH>
__global__ void __launch_bounds__(kRyserThreads, (ZO || PATH == kPathGlynn) ? 3 : 2)
ryser_int_kernel(const long long* __restrict__ mats, const ItemDesc* __restrict__ items,
                 long long total_parts, long long part0, long long item_parts,
                 const int* __restrict__ widths, int allow192, IPartial* __restrict__ partials) {
    using E = typename std::conditional<ZO, unsigned, unsigned long long>::type;
    constexpr int NP = ZO ? ((N + 3) & ~3) : ((N + 1) & ~1);   // 16-byte columns
    constexpr bool kEq4 = !ZO && PATH != kPathGlynn;            // Eq. (4) codes needed
    __shared__ __align__(16) E s_col[kEq4 ? N * NP : 1];        // s_col[j * NP + i] = a_ij
    __shared__ __align__(16) int s_col2[N * NP];                // Glynn: 2 a_ij
    __shared__ int s_row[NP];                                   // Glynn: sum_j a_ij
    __shared__ int s_cls;                                       // integers: row-sum class
    constexpr bool kBits = ZO && N >= 12 && N <= 32;            // bit-sliced Glynn walk
    using M = unsigned;
    __shared__ M s_cm[kBits ? N : 1];                           // bit i: a_ij = 1
    __shared__ M s_rm[kBits ? N : 1];                           // bit j - 1: a_ij = 1 (j >= 1)
    __shared__ M s_q[kBits ? kRyserThreads / 32 : 1][kBits ? 64 : 1];   // per-warp queues
    __shared__ unsigned long long s_acc[kAccWords][kRyserThreads];
    __shared__ int s_width;
    constexpr int G = N;
    constexpr long long kParts = (G > kLogCodesPerPart) ? (1ll << (G - kLogCodesPerPart)) : 1ll;
    constexpr int kLogPart = (G > kLogCodesPerPart) ? kLogCodesPerPart : G;
    constexpr int kLogThr = kLogPart >= 8 ? 8 : kLogPart;
    constexpr int kLogLen = kLogPart - kLogThr;
    // Glynn (0/1, widths 64 and 128): a piece holds half as many codes
    constexpr int kLogPartG = kLogPart - 1;
    constexpr int kLogThrG = kLogPartG >= 8 ? 8 : kLogPartG;
    constexpr int kLogLenG = kLogPartG - kLogThrG;
    constexpr int kL64 = (64 + N - 1 + 31) / 32, kL128 = (128 + N - 1 + 31) / 32;
    constexpr int kL192 = (192 + N - 1 + 31) / 32;
    constexpr int kMaxW = max_width<N, ZO>();
    constexpr int kG01 = glynn_group<N, N>();                   // |rho_i| <= n
    constexpr int kG1 = glynn_group<kRowBound1, N>(), kG2 = glynn_group<kRowBound2, N>();
    const long long count = total_parts / item_parts;           // widths[count + i]: row-sum class

    for (long long task = blockIdx.x; task < total_parts; task += gridDim.x) {
        const ItemDesc d = items[task / item_parts];
        const long long part = part0 + task % item_parts;           // as in ryser_c128_kernel
        const long long* a = mats + d.offset;
        __syncthreads();
        if (threadIdx.x == 0) {
            s_width = widths[task / item_parts];
            s_cls = widths[count + task / item_parts];
        }
        __syncthreads();
        const int w = s_width;
        // width computed: the decided one; past the bound, the widest the output holds
        int cw = w == kWidthInvalid ? 0 : (w == kWidthOverflow ? (allow192 ? 192 : 128) : w);
        if (cw > kMaxW) cw = kMaxW;
        if constexpr (!ZO) {
            const bool glynn = (cw == 64 || cw == 128) && s_cls != 0;
            if (glynn != (PATH == kPathGlynn)) continue;     // the other launch's item (uniform)
        }
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int i = e / N, j = e % N;
            if constexpr (kEq4) s_col[j * NP + i] = (E)a[e];
            // exact whenever the Glynn walk runs (row sums <= 32767); unused otherwise
            s_col2[j * NP + i] = (int)(unsigned)(2ull * (unsigned long long)a[e]);
        }
        if (threadIdx.x < N) {
            unsigned long long rs = 0;
            for (int j = 0; j < N; j++) rs += (unsigned long long)a[threadIdx.x * N + j];
            s_row[threadIdx.x] = (int)(unsigned)rs;
        }
        if constexpr (kBits) {
            if (threadIdx.x < N) {
                const int t = threadIdx.x;
                M cm = 0, rm = 0;
                for (int i = 0; i < N; i++) cm |= (M)(a[i * N + t] != 0 ? 1u : 0u) << i;
                for (int j = 1; j < N; j++) rm |= (M)(a[t * N + j] != 0 ? 1u : 0u) << (j - 1);
                s_cm[t] = cm;
                s_rm[t] = rm;
            }
        }
        __syncthreads();
        int shift = 0;                  // Glynn: the sum is 2^(n-1) per(A)
        AccWords acc = {0ull, 0ull, 0ull, 0ull};
        if constexpr (ZO) {
            if (cw > 0) {               // every width by Glynn's form
                shift = N - 1;
                if (threadIdx.x < (1 << kLogThrG)) {
                    const unsigned long long g0 = ((unsigned long long)part << kLogPartG) +
                                                  ((unsigned long long)threadIdx.x << kLogLenG);
                    if constexpr (kBits) {
                        // every thread of the CTA takes part (kLogThrG = 8): full warps
                        M* q = s_q[threadIdx.x >> 5];
                        if (cw == 64) glynn_bits_range<N, kL64, M>(s_cm, s_rm, s_row, q, (M)g0, kLogLenG, acc);
                        if constexpr (kMaxW >= 128) {
                            if (cw == 128)
                                glynn_bits_range<N, kL128, M>(s_cm, s_rm, s_row, q, (M)g0, kLogLenG, acc);
                        }
                    } else {
                        if (cw == 64) glynn_range<N, NP, kL64, kG01>(s_col2, s_row, g0, kLogLenG, acc);
                        if constexpr (kMaxW >= 128) {
                            if (cw == 128) glynn_range<N, NP, kL128, kG01>(s_col2, s_row, g0, kLogLenG, acc);
                        }
                        if constexpr (kMaxW >= 192) {
                            if (cw == 192) glynn_range<N, NP, kL192, kG01>(s_col2, s_row, g0, kLogLenG, acc);
                        }
                    }
                }
            }
        } else if constexpr (PATH == kPathGlynn) {
            // other integers with small row sums: the same exact Glynn walk
            const int cls = s_cls;
            if ((cw == 64 || cw == 128) && cls != 0) {
                shift = N - 1;
                if (threadIdx.x < (1 << kLogThrG)) {
                    const unsigned long long g0 = ((unsigned long long)part << kLogPartG) +
                                                  ((unsigned long long)threadIdx.x << kLogLenG);
                    if (cls == 1) {
                        if (cw == 64) glynn_range<N, NP, kL64, kG1>(s_col2, s_row, g0, kLogLenG, acc);
                        else glynn_range<N, NP, kL128, kG1>(s_col2, s_row, g0, kLogLenG, acc);
                    } else {
                        if (cw == 64) glynn_range<N, NP, kL64, kG2>(s_col2, s_row, g0, kLogLenG, acc);
                        else glynn_range<N, NP, kL128, kG2>(s_col2, s_row, g0, kLogLenG, acc);
                    }
                }
            }
        }
        if constexpr (kEq4) {
            if (shift == 0 && threadIdx.x < (1 << kLogThr) && cw > 0) {
                const unsigned long long g0 =
                    ((unsigned long long)part << kLogPart) + ((unsigned long long)threadIdx.x << kLogLen);
                if constexpr (!ZO) {
                    if (cw == 64) ryser_int_range<N, NP, 64>(s_col, g0, kLogLen, acc);
                    if (cw == 128) ryser_int_range<N, NP, 128>(s_col, g0, kLogLen, acc);
                }
                if constexpr (kMaxW >= 192) {
                    if (cw == 192) ryser_int_range<N, NP, 192>(s_col, g0, kLogLen, acc);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kAccWords; k++) s_acc[k][threadIdx.x] = acc[k];
        __syncthreads();
        for (int h = kRyserThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                AccWords x, y;
#pragma unroll
                for (int k = 0; k < kAccWords; k++) {
                    x[k] = s_acc[k][threadIdx.x + h];
                    y[k] = s_acc[k][threadIdx.x];
                }
                words_add<kAccWords>(y, x);
#pragma unroll
                for (int k = 0; k < kAccWords; k++) s_acc[k][threadIdx.x] = y[k];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            IPartial p;
#pragma unroll
            for (int k = 0; k < kAccWords; k++) p.w[k] = s_acc[k][0];
            p.meta = (unsigned long long)(unsigned)width_status(w) | ((unsigned long long)cw << 32) |
                     ((unsigned long long)shift << 48);
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

// Sum the pieces of every integer matrix (one CTA of 128 threads per matrix;
// modular addition is exact, so the order does not matter) and write the
// out_words-word result: words above the computed width are zero.
__global__ void ryser_finish_int(const ItemDesc* items, long long parts, int count,
                                 const IPartial* partials, unsigned long long* out, int out_words,
                                 int* item_status) {
    const int it = blockIdx.x;
    if (it >= count) return;
    __shared__ unsigned long long s[kAccWords][128];
    AccWords acc = {0ull, 0ull, 0ull, 0ull};
    const long long b = (long long)it * parts, e = b + parts;
    for (long long p = b + threadIdx.x; p < e; p += blockDim.x) {
        const AccWords x = {partials[p].w[0], partials[p].w[1], partials[p].w[2], partials[p].w[3]};
        words_add<kAccWords>(acc, x);
    }
#pragma unroll
    for (int k = 0; k < kAccWords; k++) s[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int h = 64; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            AccWords x, y;
#pragma unroll
            for (int k = 0; k < kAccWords; k++) {
                x[k] = s[k][threadIdx.x + h];
                y[k] = s[k][threadIdx.x];
            }
            words_add<kAccWords>(y, x);
#pragma unroll
            for (int k = 0; k < kAccWords; k++) s[k][threadIdx.x] = y[k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long meta = partials[b].meta;   // the same for every piece of the matrix
        const int st = (int)(unsigned)(meta & 0xffffffffull);
        const int cw = (int)((meta >> 32) & 0xffffull);
        const int sh = (int)((meta >> 48) & 0xffull);
        unsigned long long v0 = s[0][0], v1 = s[1][0], v2 = s[2][0];
        if (sh > 0) {       // exact division of Glynn's sum by 2^(n-1)
            const unsigned long long v3 = s[3][0];
            v0 = (v0 >> sh) | (v1 << (64 - sh));
            v1 = (v1 >> sh) | (v2 << (64 - sh));
            v2 = (v2 >> sh) | (v3 << (64 - sh));
        }
        const int o = items[it].out_index;
        unsigned long long* dst = out + (size_t)out_words * o;
        dst[0] = cw >= 64 ? v0 : 0ull;
        dst[1] = cw >= 128 ? v1 : 0ull;
        if (out_words == 4) {
            dst[2] = cw >= 192 ? v2 : 0ull;
            dst[3] = 0ull;
        }
        if (item_status) item_status[o] = st;
    }
}

// Integer width of every matrix of a launch, once (one warp per matrix), in
// widths[i]; in widths[count + i] the row-sum class of the Glynn walk for
// general integers: 1 if every row sum is <= 127, 2 if <= 32767, else 0.
__global__ void ryser_widths_kernel(const long long* mats, const ItemDesc* items, int count, int n,
                                    int zero_one, int allow192, int* widths) {
    const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);   // uniform per warp
    if (i >= count) return;
    const long long* a = mats + items[i].offset;
    const int w = decide_width_warp(a, n, zero_one != 0, allow192 != 0);
    const int lane = threadIdx.x & 31;
    if (zero_one) {             // the class is used by general integers only
        if (lane == 0) {
            widths[i] = w;
            widths[count + i] = 0;
        }
        return;
    }
    unsigned long long rmax = 0ull;
    for (int r = lane; r < n; r += 32) {
        unsigned long long rs = 0ull;
        for (int j = 0; j < n; j++) rs += (unsigned long long)a[(size_t)r * n + j];
        rmax = rs > rmax ? rs : rmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, rmax, o);
        rmax = v > rmax ? v : rmax;
    }
    if (lane == 0) {
        widths[i] = w;
        widths[count + i] = rmax <= kRowBound1 ? 1 : (rmax <= kRowBound2 ? 2 : 0);
    }
}

template <int N>
cudaError_t launch_n(int dtype, const void* mats, const ItemDesc* items, long long total_parts,
                     long long part0, long long item_parts,
                     const int* widths, int allow192, void* partials, int grid, cudaStream_t st) {
    const int g = (int)std::min<long long>(total_parts, (long long)grid);
    if (dtype == PERM_C128) {
        ryser_c128_kernel<N><<<g, kRyserThreads, 0, st>>>((const double2*)mats, items, total_parts, part0,
                                                          item_parts,
                                                          (CPartial*)partials);
    } else if (dtype == PERM_U01) {
        ryser_int_kernel<N, true, kPathAll><<<g, kRyserThreads, 0, st>>>(
            (const long long*)mats, items, total_parts, part0, item_parts, widths, allow192,
            (IPartial*)partials);
    } else {
        ryser_int_kernel<N, false, kPathGlynn><<<g, kRyserThreads, 0, st>>>(
            (const long long*)mats, items, total_parts, part0, item_parts, widths, allow192,
            (IPartial*)partials);
        ryser_int_kernel<N, false, kPathEq4><<<g, kRyserThreads, 0, st>>>(
            (const long long*)mats, items, total_parts, part0, item_parts, widths, allow192,
            (IPartial*)partials);
    }
    return cudaGetLastError();
}

typedef cudaError_t (*launch_fn)(int, const void*, const ItemDesc*, long long, long long, long long,
                                 const int*, int, void*, int, cudaStream_t);

// Load the kernels of order N for `dtype` now (cudaFuncGetAttributes makes the
// runtime load a function): a lazy load at the first launch can wait for every
// kernel running on the device, which would stall a serving thread.
template <int N>
cudaError_t preload_n(int dtype) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (dtype == PERM_C128) {
        e = cudaFuncGetAttributes(&fa, (const void*)ryser_c128_kernel<N>);
    } else if (dtype == PERM_U01) {
        e = cudaFuncGetAttributes(&fa, (const void*)ryser_int_kernel<N, true, kPathAll>);
    } else {
        e = cudaFuncGetAttributes(&fa, (const void*)ryser_int_kernel<N, false, kPathGlynn>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)ryser_int_kernel<N, false, kPathEq4>);
    }
    return e;
}
typedef cudaError_t (*preload_fn)(int);

template <int... Ns>
struct Table {
    static constexpr launch_fn fns[sizeof...(Ns)] = {&launch_n<Ns>...};
    static constexpr preload_fn pre[sizeof...(Ns)] = {&preload_n<Ns>...};
};

#define PERM_NS 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, \
                24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40
using NTable = Table<PERM_NS>;

}  // namespace


// Launch Ryser for `count` matrices that all have order n (1 <= n <= 40);
// `partials` holds count * ryser_parts(dtype, n) slots of ryser_partial_bytes(dtype)
// and `widths` 2 * count ints (integer types only).
cudaError_t ryser_launch_group(int dtype, int n, const void* mats, const ItemDesc* items, int count,
                               void* partials, int* widths, void* out, int out_words, bool allow192,
                               int* item_status, int grid, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (n < 1 || n > kMaxN) return cudaErrorInvalidValue;
    if (dtype != PERM_C128 && out_words != 2 && out_words != 4) return cudaErrorInvalidValue;
    if (allow192 && out_words != 4) return cudaErrorInvalidValue;
    const long long parts = parts_for(dtype, n);
    if (dtype != PERM_C128) {
        ryser_widths_kernel<<<(count + 3) / 4, 128, 0, st>>>((const long long*)mats, items, count, n,
                                                                 dtype == PERM_U01, allow192 ? 1 : 0,
                                                                 widths);
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = NTable::fns[n - 1](dtype, mats, items, (long long)count * parts, 0ll, parts, widths,
                                       allow192 ? 1 : 0, partials, grid, st);
    if (e != cudaSuccess) return e;
    if (dtype == PERM_C128)
        ryser_finish_c128<<<count, 32, 0, st>>>(items, parts, count, (const CPartial*)partials,
                                                (double2*)out, item_status);
    else
        ryser_finish_int<<<count, 128, 0, st>>>(items, parts, count, (const IPartial*)partials,
                                                (unsigned long long*)out, out_words, item_status);
    return cudaGetLastError();
}

// Pieces [begin, end) of one matrix's codes (item: one device descriptor), their
// partial sums written to partials[0 .. end - begin).  The pieces are the ones
// ryser_launch_group cuts, so the sums are the same bits.
cudaError_t ryser_launch_pieces(int dtype, int n, const void* mats, const ItemDesc* item, long long begin,
                                long long end, void* partials, int* widths, bool allow192, int grid,
                                cudaStream_t st) {
    if (n < 1 || n > kMaxN || begin < 0 || end > parts_for(dtype, n) || begin > end)
        return cudaErrorInvalidValue;
    if (begin == end) return cudaSuccess;
    if (dtype != PERM_C128) {
        ryser_widths_kernel<<<1, 128, 0, st>>>((const long long*)mats, item, 1, n, dtype == PERM_U01,
                                               allow192 ? 1 : 0, widths);
        const cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    return NTable::fns[n - 1](dtype, mats, item, end - begin, begin, end - begin, widths, allow192 ? 1 : 0,
                              partials, grid, st);
}

// The finishing kernel of one matrix over all of its pieces' partial sums.
cudaError_t ryser_finish_one(int dtype, int n, const ItemDesc* item, const void* partials, void* out,
                             int out_words, int* item_status, cudaStream_t st) {
    if (n < 1 || n > kMaxN) return cudaErrorInvalidValue;
    const long long parts = parts_for(dtype, n);
    if (dtype == PERM_C128)
        ryser_finish_c128<<<1, 32, 0, st>>>(item, parts, 1, (const CPartial*)partials, (double2*)out,
                                            item_status);
    else
        ryser_finish_int<<<1, 128, 0, st>>>(item, parts, 1, (const IPartial*)partials,
                                            (unsigned long long*)out, out_words, item_status);
    return cudaGetLastError();
}

long long ryser_parts(int dtype, int n) { return parts_for(dtype, n); }

size_t ryser_partial_bytes(int dtype) { return dtype == PERM_C128 ? sizeof(CPartial) : sizeof(IPartial); }

cudaError_t ryser_preload(int dtype, int n_max) {
    cudaFuncAttributes fa;
    cudaError_t e = dtype == PERM_C128 ? cudaFuncGetAttributes(&fa, (const void*)ryser_finish_c128)
                                       : cudaFuncGetAttributes(&fa, (const void*)ryser_finish_int);
    if (e == cudaSuccess && dtype != PERM_C128) e = cudaFuncGetAttributes(&fa, (const void*)ryser_widths_kernel);
    for (int n = 1; n <= std::min(n_max, kMaxN) && e == cudaSuccess; n++) e = NTable::pre[n - 1](dtype);
    return e;
}

}  // namespace perm
