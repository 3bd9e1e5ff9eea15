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
                u = __fma_rn(P2, -1.0, P1);
                v = __fma_rn(P2, -1.0, __fma_rn(P1, -1.0, P3));
                w = __fma_rn(u, 1.0, v);
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
