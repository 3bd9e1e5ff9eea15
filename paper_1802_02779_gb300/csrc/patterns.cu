// patterns.cu -- all collision-free output patterns in one Store-zechin pass.
//
// For boson sampling (Su & Zheng, arXiv:1802.02779, Section 2) the amplitude of
// an output pattern is the permanent of the r x r submatrix of the r input rows
// of U and the pattern's r output columns.  Store-zechin's stored
// sub-permanents (Section 4) are per(rows 0..k-1, columns S) for column sets S;
// run on the r x c matrix of the input rows over all c output columns, its
// level r holds per(rows 0..r-1, S) for every r-subset S of the columns, i.e.
// the amplitudes of all C(c, r) collision-free patterns, in one pass instead of
// C(c, r) separate permanents (space for time, Section 6).  The paper does not
// do this; it is the same recurrence, stopped at level r.
//
// One CTA per input matrix, the whole table in shared memory (c <= 13).  The
// entries of level k are in colex order of their column sets and every entry
// is summed in ascending column order exactly like the square kernels, with
// the three-multiplication complex form below level r and a double-double
// four-product sum at level r -- so every pattern's value is bit-identical to
// perm_batch on that pattern's r x r submatrix.
#include "perm_internal.cuh"

namespace perm {
namespace {

constexpr int kPatMaxCols = 13;
constexpr int kPatThreads = 256;

// Shared-memory layout: every piece starts on a 16-byte boundary (double2 accesses).
struct PatLayout { int cxy, cs, suv, sw, total; };
__host__ __device__ inline int pat_align16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline PatLayout pat_layout(int rows, int cols) {
    PatLayout L;
    L.cxy = 0;
    L.cs = pat_align16(L.cxy + 16 * rows * cols);
    L.suv = pat_align16(L.cs + 8 * rows * cols);
    L.sw = pat_align16(L.suv + 16 * (1 << cols));
    L.total = pat_align16(L.sw + 8 * (1 << cols));
    return L;
}

unsigned pat_binom_host(int n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned long long r = 1;
    for (int i = 1; i <= k; i++) r = r * (unsigned long long)(n - k + i) / (unsigned long long)i;
    return (unsigned)r;
}

__device__ __forceinline__ unsigned pat_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned r = 1;
    for (int i = 1; i <= k; i++) r = r * (unsigned)(n - k + i) / (unsigned)i;
    return r;
}

// mask of the colex-rank-r l-subset of {0..c-1}
__device__ __forceinline__ unsigned pat_unrank(unsigned r, int l, int c) {
    unsigned mask = 0;
    int x = c - 1;
    for (int p = l - 1; p >= 0; p--) {
        while (pat_binom(x, p + 1) > r) x--;
        mask |= 1u << x;
        r -= pat_binom(x, p + 1);
        x--;
    }
    return mask;
}

__global__ void __launch_bounds__(kPatThreads)
patterns_c128(const double2* __restrict__ mats, int count, int rows, int cols, double2* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int item = blockIdx.x;
    if (item >= count) return;
    const double2* a = mats + (size_t)item * rows * cols;
    const unsigned CL = 1u << cols;
    const PatLayout L = pat_layout(rows, cols);
    double2* cxy = reinterpret_cast<double2*>(smem + L.cxy);     // rows * cols
    double* cs = reinterpret_cast<double*>(smem + L.cs);         // rows * cols
    double2* suv = reinterpret_cast<double2*>(smem + L.suv);     // 2^cols, by mask (16-byte aligned)
    double* sw = reinterpret_cast<double*>(smem + L.sw);
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
        const double2 z = a[e];
        cxy[e] = z;
        cs[e] = __fma_rn(z.x, 1.0, z.y);
    }
    __syncthreads();
    const unsigned nout = pat_binom(cols, rows);
    double2* o = out + (size_t)item * nout;
    for (int l = 0; l <= rows; l++) {
        const unsigned cnt = pat_binom(cols, l);
        const double2* rxy = cxy + (l >= 1 ? l - 1 : 0) * cols;
        const double* rs = cs + (l >= 1 ? l - 1 : 0) * cols;
        for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
            const unsigned mask = pat_unrank(r, l, cols);
            double u, v, w;
            if (l == 0) {
                u = 1.0; v = 0.0; w = 1.0;
            } else if (l == 1) {
                const int col = __ffs(mask) - 1;
                u = cxy[col].x; v = cxy[col].y; w = cs[col];
            } else if (l == rows) {
                dd2 re = {0.0, 0.0}, im = {0.0, 0.0};
                unsigned mm = mask;
                while (mm) {
                    const int j = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const double2 p = suv[mask ^ (1u << j)];
                    const double2 c = rxy[j];
                    re = dd_add_prod(re, c.x, p.x);
                    re = dd_add_prod(re, -c.y, p.y);
                    im = dd_add_prod(im, c.x, p.y);
                    im = dd_add_prod(im, c.y, p.x);
                }
                u = dd_round(re); v = dd_round(im); w = __dadd_rn(u, v);
            } else {
                double P1 = 0.0, P2 = 0.0, P3 = 0.0;
                unsigned mm = mask;
                while (mm) {
                    const int j = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const unsigned pm = mask ^ (1u << j);
                    const double2 p = suv[pm];
                    const double2 c = rxy[j];
                    P1 = __fma_rn(c.x, p.x, P1);
                    P2 = __fma_rn(c.y, p.y, P2);
                    P3 = __fma_rn(rs[j], sw[pm], P3);
                }
                u = __fma_rn(P2, -1.0, P1);         // the epilogue of chain_c128
                w = __fma_rn(P2, -2.0, P3);
                v = __fma_rn(u, -1.0, w);
            }
            suv[mask] = make_double2(u, v);
            sw[mask] = w;
            if (l == rows) o[r] = make_double2(u, v);
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace perm

extern "C" perm_status perm_patterns(const void* mats, int count, int rows, int cols, void* out,
                                     void* stream) {
    using namespace perm;
    if (count < 0 || rows < 1 || cols < rows || cols > kPatMaxCols) return PERM_EINVAL;
    if (count == 0) return PERM_OK;
    if (!mats || !out) return PERM_EINVAL;
    const int smem = pat_layout(rows, cols).total;
    cudaError_t e = cudaFuncSetAttribute((const void*)patterns_c128,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return PERM_ECUDA;
    patterns_c128<<<count, kPatThreads, smem, (cudaStream_t)stream>>>(
        (const double2*)mats, count, rows, cols, (double2*)out);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

// ---------------------------------------------------------------------------
// All output patterns WITH collisions (repeated output modes).
//
// An output pattern of r photons over c modes is a multiset M (mode j occupied
// t_j times, sum t_j = r); its amplitude is the permanent of the r x r matrix of
// the input rows and the columns of M with repetition, and its probability is
// |per|^2 / prod_j t_j!.  Developing along row k-1 as in Section 3.1 (property
// 4), the t_j positions that hold mode j give identical minors, so
//     T_k[M] = sum_{j in M, ascending} t_j * a[k-1][j] * T_{k-1}[M - j],
// the Store-zechin recurrence over multisets.  Multisets of size k are ranked
// through the bijection M = (m_0 <= ... <= m_{k-1})  <->  {m_i + i}, a k-subset
// of {0..c+k-2}, in colex order.  Two levels live in shared memory.
// ---------------------------------------------------------------------------
namespace perm {
namespace {

constexpr int kMsMaxEntries = 12000;     // entries (16 B each) of the two live levels

__device__ __forceinline__ unsigned ms_binom(int n, int k) { return pat_binom(n, k); }

// multiset of size k over c modes with colex rank r -> counts in `cnt` (c entries)
__device__ inline void ms_unrank(unsigned r, int k, int c, unsigned char* cnt) {
    for (int j = 0; j < c; j++) cnt[j] = 0;
    int x = c + k - 2;
    for (int p = k - 1; p >= 0; p--) {
        while (ms_binom(x, p + 1) > r) x--;
        r -= ms_binom(x, p + 1);
        cnt[x - p]++;                    // element p of the subset is m_p + p
        x--;
    }
}

// colex rank of the multiset given by counts (size k)
__device__ inline unsigned ms_rank(const unsigned char* cnt, int c) {
    unsigned r = 0;
    int p = 0;
    for (int j = 0; j < c; j++)
        for (int q = 0; q < cnt[j]; q++, p++) r += ms_binom(j + p, p + 1);
    return r;
}

__global__ void __launch_bounds__(kPatThreads)
patterns_multiset_c128(const double2* __restrict__ mats, int count, int rows, int cols,
                       double2* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int item = blockIdx.x;
    if (item >= count) return;
    const double2* a = mats + (size_t)item * rows * cols;
    const unsigned lvl_max = ms_binom(cols + rows - 1, rows);
    double2* cxy = reinterpret_cast<double2*>(smem);                      // rows * cols
    double2* buf0 = reinterpret_cast<double2*>(smem + 16 * rows * cols);   // level k-1
    double2* buf1 = buf0 + lvl_max;                                        // level k
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) cxy[e] = a[e];
    if (threadIdx.x == 0) buf0[0] = make_double2(1.0, 0.0);               // T_0 = 1
    __syncthreads();
    double2* prev = buf0;
    double2* cur = buf1;
    double2* o = out + (size_t)item * lvl_max;
    for (int k = 1; k <= rows; k++) {
        const unsigned cntk = ms_binom(cols + k - 1, k);
        const double2* rxy = cxy + (k - 1) * cols;
        for (unsigned r = threadIdx.x; r < cntk; r += blockDim.x) {
            unsigned char t[kPatMaxCols];
            ms_unrank(r, k, cols, t);
            double re = 0.0, im = 0.0;
            dd2 dre = {0.0, 0.0}, dim = {0.0, 0.0};
            for (int j = 0; j < cols; j++) {
                if (!t[j]) continue;
                t[j]--;
                const double2 p = prev[ms_rank(t, cols)];
                t[j]++;
                const double m = (double)t[j];
                const double cx = m * rxy[j].x, cy = m * rxy[j].y;   // t_j * a[k-1][j]
                if (k < rows) {
                    re = __fma_rn(cx, p.x, re);
                    re = __fma_rn(-cy, p.y, re);
                    im = __fma_rn(cx, p.y, im);
                    im = __fma_rn(cy, p.x, im);
                } else {
                    dre = dd_add_prod(dre, cx, p.x);
                    dre = dd_add_prod(dre, -cy, p.y);
                    dim = dd_add_prod(dim, cx, p.y);
                    dim = dd_add_prod(dim, cy, p.x);
                }
            }
            const double2 v = k < rows ? make_double2(re, im) : make_double2(dd_round(dre), dd_round(dim));
            cur[r] = v;
            if (k == rows) o[r] = v;
        }
        __syncthreads();
        double2* tmp = prev;
        prev = cur;
        cur = tmp;
    }
}

}  // namespace
}  // namespace perm

extern "C" perm_status perm_patterns_multiset(const void* mats, int count, int rows, int cols,
                                              void* out, void* stream) {
    using namespace perm;
    if (count < 0 || rows < 1 || cols < 1 || cols > kPatMaxCols || rows > kPatMaxCols) return PERM_EINVAL;
    const unsigned lvl_max = pat_binom_host(cols + rows - 1, rows);
    if (2ull * lvl_max > (unsigned long long)kMsMaxEntries) return PERM_EINVAL;
    if (count == 0) return PERM_OK;
    if (!mats || !out) return PERM_EINVAL;
    const int smem = 16 * rows * cols + 16 * 2 * (int)lvl_max;
    cudaError_t e = cudaFuncSetAttribute((const void*)patterns_multiset_c128,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return PERM_ECUDA;
    patterns_multiset_c128<<<count, kPatThreads, smem, (cudaStream_t)stream>>>(
        (const double2*)mats, count, rows, cols, (double2*)out);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}
