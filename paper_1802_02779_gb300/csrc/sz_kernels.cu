// sz_kernels.cu -- Store-zechin (Su & Zheng, arXiv:1802.02779, Section 4).
//
// The method develops per(A) along one row at a time without signs
// (Section 3.1, property 4) and stores every sub-permanent the first time it
// is computed so that every larger minor containing it reuses it
// (Sections 4.1-4.3).  With 0-based rows and columns and T_k[S] =
// per(rows 0..k-1, columns S):
//
//     T_1[{j}] = a[0][j],
//     T_k[S]   = sum_{j in S, ascending} a[k-1][j] * T_{k-1}[S \ {j}],   2 <= k <= n,
//     per(A)   = T_n[{0..n-1}].
//
// (The paper expands the last row first; read from the bottom up that is this
// recurrence with level k built from row k-1.)
//
// GPU organisation ("chains").  The columns are split into t = n-m outer
// columns 0..t-1 and m chain columns t..n-1.  Every set S is a pair (H, L) of
// an outer part and a chain part.  A chain is the 2^m entries (H, L) of one
// outer subset H and all chain subsets L.  The recurrence splits into
//     outer terms  h in H:  T[(H \ h, L)]  -- another chain, same L
//     chain terms  j in L:  T[(H, L \ j)]  -- the same chain, |L| one smaller
// so one CTA computes one chain in shared memory: first every entry's outer
// terms, streamed (coalesced) from the predecessor chains in global memory,
// then sub-level by sub-level (|L| = 0..m) its chain terms, gathered from
// shared memory.  Chains are processed in layers of |H| = 0..t; layer s needs
// only layer s-1.
//
// Two layouts of a chain:
//   shared memory  indexed by the bit mask of L (2^m slots), so the chain
//                  parent of (H, L) for chain column j is slot L ^ (1 << j);
//   global memory  indexed by (|L|, colex rank of L): the entries of one
//                  sub-level are contiguous, and the predecessor chains use the
//                  same order, so outer-parent reads are coalesced.
// A table (g_masks) lists the masks in the global order.
//
// Complex entries use the three-multiplication form of the complex product
// (Gauss; error analysis in Higham, "Stability of a method for multiplying
// complex matrices with three real matrix multiplications", SIMAX 13 (1992)):
// every stored entry keeps u = Re T, v = Im T and w = u + v, every matrix
// entry keeps x = Re a, y = Im a and s = x + y, and a sum of products
// sum a_j T_j is accumulated as P1 = sum x u, P2 = sum y v, P3 = sum s w, with
// Re = P1 - P2, Im = P3 - P1 - P2.  That is three FP64 FMAs per term instead
// of four; on this part the FP64 pipe is the binding resource.  The final
// level (the permanent itself) is accumulated in double-double with the
// ordinary four-product form.
//
// Integer entries are evaluated modulo 2^64 or 2^128 (exact under the bound
// chosen by decide_width); zero coefficients skip their term.
//
// Summation order for every entry: outer columns ascending, then chain
// columns ascending, i.e. all columns ascending.  The order therefore depends
// on none of m, the batch, the grid or the CTA: every kernel here gives every
// matrix the same bits.
#include "perm_internal.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace perm {

namespace {

constexpr int kBinomDim = 24;            // C(x, y) for x < 24 (t <= 21, m <= 13)
constexpr int kThreadsC128Single = 512;   // layer path, default: one CTA per SM (384: two)
constexpr int kThreadsInt = 256;          // integers: up to four CTAs per SM
constexpr int kMaskTableLen = (2 << kMaxLow) - 2;   // sum_{m=1..13} 2^m

// masks of all subsets of {0..m-1}, ordered by (popcount, value); the table
// of chain width m starts at index 2^m - 2.
__device__ unsigned short g_masks[kMaskTableLen];

__host__ __device__ inline unsigned long long binom_calc(int n, int k) {
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned long long r = 1;
    for (int i = 1; i <= k; i++) r = r * (unsigned long long)(n - k + i) / (unsigned long long)i;
    return r;
}

enum ElemKind : int { kC128 = 0, kU64 = 1, kU128 = 2 };

__host__ __device__ inline int chain_bytes_smem(int kind, int m) {
    return (kind == kC128 ? 24 : (kind == kU64 ? 8 : 16)) << m;
}
__host__ __device__ inline int coef_bytes(int kind, int n) {
    return (kind == kC128 ? 24 : 8) * n * n;
}

// Shared-memory layout, 16-byte aligned pieces.
struct SmemLayout {
    int binom_off;      // unsigned[kBinomDim][kBinomDim + 1]
    int hinfo_off;      // int[2 * kBinomDim]: predecessor slot, column
    int rowmask_off;    // unsigned[kMaxN]: low columns with a nonzero entry, per row (integers)
    int coef_off;       // C128: double2 xy[n*n] then double s[n*n]; ints: u64[n*n]
    int chain_off;      // C128: double2 uv[2^m] then double w[2^m]; u64[2^m]; ulonglong2[2^m]
    int total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int kind, int n, int m) {
    SmemLayout s;
    s.binom_off = 0;
    s.hinfo_off = align16(s.binom_off + kBinomDim * (kBinomDim + 1) * 4);
    s.rowmask_off = align16(s.hinfo_off + 2 * kBinomDim * 4);
    s.coef_off = align16(s.rowmask_off + kMaxN * 4);
    s.chain_off = align16(s.coef_off + coef_bytes(kind, n));
    s.total = align16(s.chain_off + chain_bytes_smem(kind, m));
    return s;
}

struct u128 { unsigned long long lo, hi; };

__device__ __forceinline__ u128 u128_mac(u128 acc, unsigned long long c, unsigned long long plo,
                                         unsigned long long phi) {
    // acc + c * (phi:plo)  mod 2^128
    const unsigned long long lo = c * plo;
    const unsigned long long hi = __umul64hi(c, plo) + c * phi;
    const unsigned long long nlo = acc.lo + lo;
    return {nlo, acc.hi + hi + (nlo < lo ? 1ull : 0ull)};
}
__device__ __forceinline__ u128 u128_add2(u128 acc, unsigned long long plo, unsigned long long phi) {
    const unsigned long long nlo = acc.lo + plo;
    return {nlo, acc.hi + phi + (nlo < plo ? 1ull : 0ull)};
}

// Context of one matrix inside one CTA.
struct MatCtx {
    int n, m, t;
    unsigned chain_len;          // 2^m
    const unsigned* bn;          // smem binomials
    const int* hinfo;            // smem: [0..s) predecessor slots, [kBinomDim..) columns
    const unsigned short* masks; // mask list of this m (global)
    const unsigned* rowmask;     // smem: per row, the low columns with a nonzero entry
    int out_words;               // integer result slot: 2 or 4 64-bit words
};

// Predecessor info for chain H: for the p-th outer element h_p (ascending),
// the slot of H \ h_p among the (s-1)-subsets and its matrix column h_p.
__device__ __forceinline__ void chain_setup(const MatCtx& mc, unsigned Hmask, int* hinfo) {
    if (threadIdx.x == 0) {
        int hs[kBinomDim];
        int s = 0;
        for (int h = 0; h < mc.t; h++)
            if ((Hmask >> h) & 1u) hs[s++] = h;
        const unsigned* bn = mc.bn;
        for (int p = 0; p < s; p++) {
            unsigned slot = 0;
            for (int q = 0; q < s; q++) {
                if (q < p) slot += bn[hs[q] * (kBinomDim + 1) + q + 1];
                else if (q > p) slot += bn[hs[q] * (kBinomDim + 1) + q];
            }
            hinfo[p] = (int)slot;
            hinfo[kBinomDim + p] = hs[p];          // outer column h is matrix column h
        }
    }
}

// ---------------------------------------------------------------------------
// complex128 chain.  gprev: previous layer region (chains of 3*CL doubles:
// uv plane then w plane); gdst: this chain's slot or null.
//
// Two phases.  Phase 1 (outer terms): for every entry (H, L) with 2 <= k < n
// the sum over h in H of a[k-1][h] * T[(H \ h, L)] is streamed from the
// predecessor chains in global memory -- no dependence inside the chain, so
// every load of the chain can be in flight at once -- and parked in the
// entry's shared-memory slot.  Phase 2 (chain terms): sub-level by sub-level,
// each entry continues its accumulators with the terms of its chain columns,
// read from shared memory.  Outer columns are 0..t-1 and chain columns t..n-1,
// so the accumulation order is all columns ascending.
// ---------------------------------------------------------------------------
// COMPACT (orders >= kCompactN): global chains hold the uv plane only, and the outer
// phase recomputes w = u + v for each predecessor entry it loads.  COHERENT: the
// predecessors are read through L2 only (ld.global.cg), for a kernel in which other
// CTAs of the same launch wrote them (sz_flow_c128); otherwise through the read-only
// path.
template <bool COHERENT>
__device__ __forceinline__ double2 load_pred2(const double2* p) { return COHERENT ? __ldcg(p) : __ldg(p); }
template <bool COHERENT>
__device__ __forceinline__ double load_pred(const double* p) { return COHERENT ? __ldcg(p) : __ldg(p); }

template <bool COMPACT, bool COHERENT = false>
__device__ void chain_c128(const MatCtx& mc, int s, unsigned char* chain_smem, const double* gprev,
                           double* gdst, const unsigned char* coef_smem, bool last, double2* out,
                           int out_index) {
    const int n = mc.n, m = mc.m, t = mc.t;
    const unsigned CL = mc.chain_len;
    double2* suv = reinterpret_cast<double2*>(chain_smem);
    double* sw = reinterpret_cast<double*>(chain_smem + 16 * CL);
    const double2* cxy = reinterpret_cast<const double2*>(coef_smem);
    const double* cs = reinterpret_cast<const double*>(coef_smem + 16 * n * n);
    const unsigned* bn = mc.bn;
    constexpr bool compact = COMPACT;
    const size_t cwd = (compact ? 2 : 3) * (size_t)CL;          // doubles per global chain
    const int* hslot = mc.hinfo;
    const int* hcol = mc.hinfo + kBinomDim;
    const unsigned short* masks = mc.masks;

    // ---- phase 1: outer terms ----
    if (s >= 1) {
        for (unsigned idx = threadIdx.x; idx < CL; idx += blockDim.x) {
            const unsigned mask = masks[idx];
            const int k = s + __popc(mask);
            if (k < 2 || k >= n) continue;
            const double2* rxy = cxy + (k - 1) * n;
            const double* rs = cs + (k - 1) * n;
            double P1 = 0.0, P2 = 0.0, P3 = 0.0;
            for (int q = 0; q < s; q += 4) {
                double2 huv[4];
                double hw[4];
#pragma unroll
                for (int z = 0; z < 4; z++) {
                    if (q + z < s) {
                        const double* pc = gprev + (size_t)hslot[q + z] * cwd;
                        huv[z] = load_pred2<COHERENT>(reinterpret_cast<const double2*>(pc) + idx);
                        // compact tables: w = u + v, rounded once, recomputed here
                        hw[z] = compact ? __fma_rn(huv[z].x, 1.0, huv[z].y) : load_pred<COHERENT>(pc + 2 * CL + idx);
                    }
                }
#pragma unroll
                for (int z = 0; z < 4; z++) {
                    if (q + z < s) {
                        const int col = hcol[q + z];
                        const double2 c = rxy[col];
                        P1 = __fma_rn(c.x, huv[z].x, P1);
                        P2 = __fma_rn(c.y, huv[z].y, P2);
                        P3 = __fma_rn(rs[col], hw[z], P3);
                    }
                }
            }
            suv[mask] = make_double2(P1, P2);
            sw[mask] = P3;
        }
        __syncthreads();
    }

    // ---- phase 2: chain terms, sub-level by sub-level ----
    unsigned off = 0;
    for (int l = 0; l <= m; l++) {
        const unsigned cnt = bn[m * (kBinomDim + 1) + l];
        const int k = s + l;
        const int row = k >= 1 ? k - 1 : 0;
        const double2* rxy = cxy + row * n + t;      // chain column j is matrix column t + j
        const double* rs = cs + row * n + t;
        for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
            const unsigned idx = off + r;
            const unsigned mask = masks[idx];
            double u, v, w;
            if (k == 0) {
                u = 1.0; v = 0.0; w = 1.0;
            } else if (k == 1) {
                const int col = (l == 1) ? t + __ffs(mask) - 1 : hcol[0];
                u = cxy[col].x; v = cxy[col].y; w = cs[col];
            } else if (k == n) {
                // the permanent: double-double, four-product complex form, outer terms first
                const double2* fxy = cxy + (n - 1) * n;
                dd2 re = {0.0, 0.0}, im = {0.0, 0.0};
                for (int q = 0; q < s; q++) {
                    const double2 p = load_pred2<COHERENT>(reinterpret_cast<const double2*>(gprev + (size_t)hslot[q] * cwd) + idx);
                    const double2 c = fxy[hcol[q]];
                    re = dd_add_prod(re, c.x, p.x);
                    re = dd_add_prod(re, -c.y, p.y);
                    im = dd_add_prod(im, c.x, p.y);
                    im = dd_add_prod(im, c.y, p.x);
                }
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
                if (s >= 1) {                 // outer terms from phase 1
                    const double2 p = suv[mask];
                    P1 = p.x; P2 = p.y; P3 = sw[mask];
                }
                unsigned mm = mask;
                while (mm) {
                    const int j = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const unsigned pm = mask ^ (1u << j);
                    const double2 p = suv[pm];
                    const double pw = sw[pm];
                    const double2 c = rxy[j];
                    P1 = __fma_rn(c.x, p.x, P1);
                    P2 = __fma_rn(c.y, p.y, P2);
                    P3 = __fma_rn(rs[j], pw, P3);
                }
                // Re = P1 - P2 and w = Re + Im = P3 - 2 P2 (one rounding each),
                // Im = w - Re: three FP64 operations, written as FMAs with
                // constant factors (the pipe issues FMAs faster than adds)
                u = __fma_rn(P2, -1.0, P1);
                w = __fma_rn(P2, -2.0, P3);
                v = __fma_rn(u, -1.0, w);
            }
            suv[mask] = make_double2(u, v);
            sw[mask] = w;
            if (gdst) {
                reinterpret_cast<double2*>(gdst)[idx] = make_double2(u, v);
                if (!compact) gdst[2 * CL + idx] = w;
            }
            if (last && l == m) out[out_index] = make_double2(u, v);
        }
        off += cnt;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// integer chain modulo 2^64 (W128 = false) or 2^128 (W128 = true), same two
// phases.  ZO: coefficients are 0/1 (add instead of multiply-add).  Global
// chain: CL words (u64) or CL ulonglong2 (u128).
// ---------------------------------------------------------------------------
template <bool W128, bool ZO>
__device__ void chain_int(const MatCtx& mc, int s, unsigned char* chain_smem,
                          const unsigned long long* gprev, unsigned long long* gdst,
                          const unsigned long long* coef, bool last, unsigned long long* out,
                          int out_index) {
    const int n = mc.n, m = mc.m, t = mc.t;
    const unsigned CL = mc.chain_len;
    const unsigned* bn = mc.bn;
    const int* hslot = mc.hinfo;
    const int* hcol = mc.hinfo + kBinomDim;
    const unsigned short* masks = mc.masks;
    constexpr int kW = W128 ? 2 : 1;     // words per entry
    unsigned long long* sv = reinterpret_cast<unsigned long long*>(chain_smem);
    ulonglong2* sv2 = reinterpret_cast<ulonglong2*>(chain_smem);

    // ---- phase 1: outer terms (zero coefficients skipped; a uniform test) ----
    if (s >= 1) {
        for (unsigned idx = threadIdx.x; idx < CL; idx += blockDim.x) {
            const unsigned mask = masks[idx];
            const int k = s + __popc(mask);
            if (k < 2) continue;
            const unsigned long long* rc = coef + (k - 1) * n;
            u128 val = {0ull, 0ull};
            for (int q = 0; q < s; q += 4) {
                unsigned long long hlo[4], hhi[4], hc[4];
#pragma unroll
                for (int z = 0; z < 4; z++) {
                    hlo[z] = 0ull; hhi[z] = 0ull;
                    hc[z] = (q + z < s) ? rc[hcol[q + z]] : 0ull;
                    if (hc[z] != 0ull) {
                        const unsigned long long* pc = gprev + (size_t)hslot[q + z] * kW * CL;
                        if (W128) {
                            const ulonglong2 p = __ldg(reinterpret_cast<const ulonglong2*>(pc) + idx);
                            hlo[z] = p.x; hhi[z] = p.y;
                        } else {
                            hlo[z] = __ldg(pc + idx);
                        }
                    }
                }
#pragma unroll
                for (int z = 0; z < 4; z++) {
                    if (hc[z] != 0ull) {
                        if (W128) val = ZO ? u128_add2(val, hlo[z], hhi[z]) : u128_mac(val, hc[z], hlo[z], hhi[z]);
                        else val.lo += ZO ? hlo[z] : hc[z] * hlo[z];
                    }
                }
            }
            if (W128) sv2[mask] = make_ulonglong2(val.lo, val.hi);
            else sv[mask] = val.lo;
        }
        __syncthreads();
    }

    // ---- phase 2: chain terms ----
    unsigned off = 0;
    for (int l = 0; l <= m; l++) {
        const unsigned cnt = bn[m * (kBinomDim + 1) + l];
        const int k = s + l;
        const unsigned long long* rc = coef + (k >= 1 ? (k - 1) * n : 0) + t;
        const unsigned rmask = k >= 1 ? mc.rowmask[k - 1] : 0u;
        for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
            const unsigned idx = off + r;
            const unsigned mask = masks[idx];
            u128 val = {0ull, 0ull};
            if (k == 0) {
                val.lo = 1ull;
            } else if (k == 1) {
                const int col = (l == 1) ? t + __ffs(mask) - 1 : hcol[0];
                val.lo = coef[col];
            } else {
                if (s >= 1) {                 // outer terms from phase 1
                    if (W128) { const ulonglong2 p = sv2[mask]; val.lo = p.x; val.hi = p.y; }
                    else val.lo = sv[mask];
                }
                // chain terms: only the columns of L whose coefficient is nonzero
                unsigned mm = mask & rmask;
                while (mm) {
                    const int j = __ffs(mm) - 1;
                    mm &= mm - 1;
                    const unsigned pm = mask ^ (1u << j);
                    if (W128) {
                        const ulonglong2 p = sv2[pm];
                        val = ZO ? u128_add2(val, p.x, p.y) : u128_mac(val, rc[j], p.x, p.y);
                    } else {
                        val.lo += ZO ? sv[pm] : rc[j] * sv[pm];
                    }
                }
            }
            if (W128) {
                sv2[mask] = make_ulonglong2(val.lo, val.hi);
                if (gdst) reinterpret_cast<ulonglong2*>(gdst)[idx] = make_ulonglong2(val.lo, val.hi);
            } else {
                sv[mask] = val.lo;
                if (gdst) gdst[idx] = val.lo;
            }
            if (last && l == m) {
                unsigned long long* dst = out + (size_t)mc.out_words * out_index;
                dst[0] = val.lo;
                dst[1] = W128 ? val.hi : 0ull;
                if (mc.out_words == 4) { dst[2] = 0ull; dst[3] = 0ull; }
            }
        }
        off += cnt;
        __syncthreads();
    }
}

// Colex unranking of an s-subset of {0..t-1} (uniform, one thread).
__device__ inline unsigned unrank_high(unsigned slot, int s, int t, const unsigned* bn) {
    unsigned mask = 0;
    int c = t - 1;
    for (int p = s - 1; p >= 0; p--) {
        while (bn[c * (kBinomDim + 1) + p + 1] > slot) c--;
        mask |= 1u << c;
        slot -= bn[c * (kBinomDim + 1) + p + 1];
        c--;
    }
    return mask;
}

__device__ inline void fill_binom(unsigned* bn) {
    for (int e = threadIdx.x; e < kBinomDim * (kBinomDim + 1); e += blockDim.x) {
        const int x = e / (kBinomDim + 1), y = e % (kBinomDim + 1);
        bn[e] = (unsigned)binom_calc(x, y);
    }
}

// Load the coefficients of one matrix into shared memory.
__device__ inline void load_coef_c128(const double2* a, int n, unsigned char* coef) {
    double2* xy = reinterpret_cast<double2*>(coef);
    double* sm = reinterpret_cast<double*>(coef + 16 * n * n);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const double2 z = a[e];
        xy[e] = z;
        sm[e] = __fma_rn(z.x, 1.0, z.y);
    }
}
__device__ inline void load_coef_int(const long long* a, int n, int m, unsigned long long* coef,
                                     unsigned* rowmask) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) coef[e] = (unsigned long long)a[e];
    const int t = n - m;                       // chain column j is matrix column t + j
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        unsigned rm = 0;
        for (int j = 0; j < m; j++)
            if (a[(size_t)i * n + t + j] != 0) rm |= 1u << j;
        rowmask[i] = rm;
    }
}

__device__ inline void init_ctx(MatCtx& mc, int n, int m_param, const unsigned char* smem,
                                const SmemLayout& L) {
    mc.n = n;
    mc.m = sz_low_for(n, m_param);
    mc.t = n - mc.m;
    mc.chain_len = 1u << mc.m;
    mc.bn = reinterpret_cast<const unsigned*>(smem + L.binom_off);
    mc.hinfo = reinterpret_cast<const int*>(smem + L.hinfo_off);
    mc.masks = g_masks + ((1 << mc.m) - 2);
    mc.rowmask = reinterpret_cast<const unsigned*>(smem + L.rowmask_off);
    mc.out_words = 2;
}

// Global-memory words of one chain (complex: 2 per entry in compact tables, else 3).
__host__ __device__ inline size_t chain_words(int kind, int m, bool compact = false) {
    return (size_t)(kind == kC128 ? (compact ? 2 : 3) : (kind == kU64 ? 1 : 2)) << m;
}

// One chain of a matrix, any element kind (COMPACT, COHERENT: see chain_c128).
template <int KIND, bool ZO, bool COMPACT = false, bool COHERENT = false>
__device__ __forceinline__ void run_chain(const MatCtx& mc, int s, unsigned char* smem_chain,
                                          const unsigned long long* src, unsigned long long* dst,
                                          const unsigned char* coef, bool last, void* out,
                                          int out_index) {
    if (KIND == kC128)
        chain_c128<COMPACT, COHERENT>(mc, s, smem_chain, reinterpret_cast<const double*>(src),
                   reinterpret_cast<double*>(dst), coef, last, reinterpret_cast<double2*>(out),
                   out_index);
    else
        chain_int<KIND == kU128, ZO>(mc, s, smem_chain, src, dst,
                                     reinterpret_cast<const unsigned long long*>(coef), last,
                                     reinterpret_cast<unsigned long long*>(out), out_index);
}

// All chains of one matrix, inside one CTA (batched mode).  ws: this CTA's
// workspace, two layer regions of C(t, t/2) chains each.
template <int KIND, bool ZO>
__device__ void run_matrix_cta(const MatCtx& mc, unsigned char* smem_chain, unsigned long long* ws,
                               const unsigned char* coef, void* out, int out_index, int* hinfo) {
    const size_t CW = chain_words(KIND, mc.m);     // batched matrices are below kCompactN
    const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * CW;
    for (int s = 0; s <= mc.t; s++) {
        const unsigned nslots = (unsigned)binom_calc(mc.t, s);
        unsigned long long* dst_region = ws + (size_t)(s & 1) * layer_words;
        const unsigned long long* src_region = ws + (size_t)((s + 1) & 1) * layer_words;
        const bool last = (s == mc.t);
        for (unsigned slot = 0; slot < nslots; slot++) {
            chain_setup(mc, unrank_high(slot, s, mc.t, mc.bn), hinfo);
            __syncthreads();
            run_chain<KIND, ZO>(mc, s, smem_chain, src_region,
                                last ? nullptr : dst_region + (size_t)slot * CW, coef, last, out,
                                out_index);
            // every chain ends with __syncthreads()
        }
    }
}

// ---------------------------------------------------------------------------
// Batched kernels: one CTA per matrix, persistent over the item list.
// ---------------------------------------------------------------------------
template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS <= 384 ? 2 : 1)
sz_batched_c128(const double2* __restrict__ mats, const ItemDesc* __restrict__ items, int count,
                int m_param, double2* out, int* item_status, unsigned long long* workspace,
                size_t ws_words_per_cta, unsigned* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    fill_binom(reinterpret_cast<unsigned*>(smem));
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= count) break;
        const ItemDesc d = items[it];
        const int n = d.n;
        const SmemLayout L = smem_layout(kC128, n, sz_low_for(n, m_param));
        MatCtx mc;
        init_ctx(mc, n, m_param, smem, L);
        load_coef_c128(mats + d.offset, n, smem + L.coef_off);
        __syncthreads();
        run_matrix_cta<kC128, false>(mc, smem + L.chain_off,
                                     workspace + (size_t)blockIdx.x * ws_words_per_cta,
                                     smem + L.coef_off, out, d.out_index,
                                     reinterpret_cast<int*>(smem + L.hinfo_off));
        if (item_status && threadIdx.x == 0) item_status[d.out_index] = PERM_OK;
    }
}

// W64ONLY: the host guarantees every item fits 64 bits (0/1 input, n <= 20),
// so the chain needs only one word per entry.  THREADS: 256 (up to four CTAs
// per SM) or 512 (two).
template <bool ZO, bool W64ONLY, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 3 : 2)
sz_batched_int(const long long* __restrict__ mats, const ItemDesc* __restrict__ items, int count,
               int m_param, unsigned long long* out, int out_words, int* item_status,
               unsigned long long* workspace, size_t ws_words_per_cta, unsigned* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ int s_width;
    fill_binom(reinterpret_cast<unsigned*>(smem));
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= count) break;
        const ItemDesc d = items[it];
        const int n = d.n;
        if (threadIdx.x == 0) s_width = decide_width(mats + d.offset, n, ZO);
        const SmemLayout L = smem_layout(W64ONLY ? kU64 : kU128, n, sz_low_for(n, m_param));
        MatCtx mc;
        init_ctx(mc, n, m_param, smem, L);
        mc.out_words = out_words;
        unsigned long long* coef = reinterpret_cast<unsigned long long*>(smem + L.coef_off);
        load_coef_int(mats + d.offset, n, mc.m, coef, reinterpret_cast<unsigned*>(smem + L.rowmask_off));
        __syncthreads();
        const int w = s_width;
        unsigned long long* ws = workspace + (size_t)blockIdx.x * ws_words_per_cta;
        int* hinfo = reinterpret_cast<int*>(smem + L.hinfo_off);
        if (W64ONLY || w == kWidth64)
            run_matrix_cta<kU64, ZO>(mc, smem + L.chain_off, ws, smem + L.coef_off, out, d.out_index, hinfo);
        else
            run_matrix_cta<kU128, ZO>(mc, smem + L.chain_off, ws, smem + L.coef_off, out, d.out_index, hinfo);
        if (item_status && threadIdx.x == 0) item_status[d.out_index] = width_status(w);
    }
}

// ---------------------------------------------------------------------------
// 0/1 matrices modulo 2^64 (every 0/1 matrix of order <= 20: 20! < 2^64) with
// register rows.  The 2^m entries of a chain are grouped into rows of 2^RB
// entries that differ only in the RB lowest chain columns ("lo"); the other
// h = m - RB chain columns ("hi") name the row.
//
// Phase 1 (outer terms) is chain_int's, two entries per thread and load.
// Phase 2 walks the rows in h + 1 stages by popcount(hi), one barrier per
// stage: a thread takes a row, adds for every hi column i of the row the row
// hi \ i (finished in an earlier stage, read from shared memory), then the
// terms inside the row in registers, in increasing lo, so that every entry
// it reads is complete.  Each entry sums exactly the terms of the §4
// recurrence, T[S] = sum over j in S with a[|S|-1][j] = 1 of T[S \ j]; only
// the order of the additions differs from chain_int, which modulo 2^64
// changes nothing.
//
// Shared memory: E, 2^m u64 by row, row hi as 2^(RB-1) 16-byte pairs, pair z
// stored at z ^ swz(hi) so that the rows a quarter warp reads together fall
// on different banks.  Global chain: natural order of the chain mask
// c = hi * 2^RB + lo.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int popc_const(int x) { return x ? (x & 1) + popc_const(x >> 1) : 0; }

template <int RB>
__device__ __forceinline__ unsigned zo_pair(unsigned hi, unsigned z) {
    constexpr unsigned kPairs = 1u << (RB - 1);
    return hi * kPairs + (z ^ ((hi >> (4 - RB)) & (kPairs - 1)));
}

// Per chain H (s outer columns, every thread passes the same H): pslot[p], the
// slot of H minus its p-th column among the (s-1)-subsets (colex rank), and
// obits[k] for k = s..s+m, bit p set when a[k-1][p-th column of H] != 0.
__device__ __forceinline__ void zo_chain_setup(const MatCtx& mc, const unsigned long long* coef,
                                               unsigned H, int s, int* pslot, unsigned* obits) {
    const unsigned* bn = mc.bn;
    const int x = (int)threadIdx.x;
    if (x < s) {
        unsigned slot = 0;
        int q = 0;
        for (unsigned hm = H; hm; hm &= hm - 1, q++) {
            const int b = __ffs(hm) - 1;
            if (q < x) slot += bn[b * (kBinomDim + 1) + q + 1];
            else if (q > x) slot += bn[b * (kBinomDim + 1) + q];
        }
        pslot[x] = (int)slot;
    } else if (x >= 32 && x - 32 <= mc.m) {
        const int k = s + (x - 32);
        unsigned bits = 0;
        if (k >= 1) {
            int p = 0;
            for (unsigned hm = H; hm; hm &= hm - 1, p++)
                if (coef[(size_t)(k - 1) * mc.n + (__ffs(hm) - 1)] != 0ull) bits |= 1u << p;
        }
        obits[k] = bits;
    }
}

template <int RB>
__device__ void chain_zo64(const MatCtx& mc, int s, ulonglong2* E, const unsigned long long* gprev,
                           unsigned long long* gdst, const int* pslot, const unsigned* obits,
                           bool last, unsigned long long* out, int out_index) {
    constexpr int kRow = 1 << RB, kPairs = kRow / 2;
    const int m = mc.m, h = m - RB;
    const unsigned CL = 1u << m;

    // ---- phase 1: outer terms, entries c and c + 1 (c even) per thread ----
    if (s >= 1) {
        unsigned po[8];                          // first eight predecessor chains (a layer region
#pragma unroll                                   // of at most 2^19 words for orders <= 20)
        for (int z = 0; z < 8; z++) po[z] = (unsigned)pslot[z < s ? z : 0] * CL;
        for (unsigned e = threadIdx.x; e < CL / 2; e += blockDim.x) {
            const unsigned c = 2 * e;
            const int k = s + __popc(c);
            const unsigned ob0 = obits[k], ob1 = obits[k + 1];
            const unsigned ob = ob0 | ob1;
            unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
            for (int z0 = 0; z0 < 8; z0 += 4) {
                if (z0 < s) {
                    ulonglong2 v[4];
#pragma unroll
                    for (int z = 0; z < 4; z++) {
                        v[z] = make_ulonglong2(0ull, 0ull);
                        if ((ob >> (z0 + z)) & 1u)
                            v[z] = __ldg(reinterpret_cast<const ulonglong2*>(gprev + po[z0 + z] + c));
                    }
#pragma unroll
                    for (int z = 0; z < 4; z++) {
                        if ((ob0 >> (z0 + z)) & 1u) a0 += v[z].x;
                        if ((ob1 >> (z0 + z)) & 1u) a1 += v[z].y;
                    }
                }
            }
            for (int p = 8; p < s; p++) {        // more than eight outer columns
                if ((ob >> p) & 1u) {
                    const ulonglong2 w =
                        __ldg(reinterpret_cast<const ulonglong2*>(gprev + (size_t)pslot[p] * CL + c));
                    if ((ob0 >> p) & 1u) a0 += w.x;
                    if ((ob1 >> p) & 1u) a1 += w.y;
                }
            }
            E[zo_pair<RB>(c >> RB, (c & (kRow - 1)) >> 1)] = make_ulonglong2(a0, a1);
        }
        __syncthreads();
    }

    // ---- phase 2: rows by popcount(hi) ----
    const unsigned short* rows = g_masks + ((1u << h) - 2);
    const unsigned full = (1u << h) - 1;
    unsigned off = 0;
    for (int q = 0; q <= h; q++) {
        const unsigned cnt = mc.bn[h * (kBinomDim + 1) + q];
        const int kr = s + q;                    // level of the row's entry lo = 0
        unsigned R[RB + 1];
        unsigned any = 0;
#pragma unroll
        for (int p = 0; p <= RB; p++) {
            R[p] = (kr + p >= 1) ? mc.rowmask[kr + p - 1] : 0u;
            any |= R[p];
        }
        any >>= RB;
        for (unsigned rr = threadIdx.x; rr < cnt; rr += blockDim.x) {
            const unsigned hi = rows[off + rr];
            unsigned long long v[kRow];
            if (s >= 1) {
#pragma unroll
                for (int z = 0; z < kPairs; z++) {
                    const ulonglong2 x = E[zo_pair<RB>(hi, z)];
                    v[2 * z] = x.x;
                    v[2 * z + 1] = x.y;
                }
            } else {
#pragma unroll
                for (int lo = 0; lo < kRow; lo++) v[lo] = 0ull;
                if (hi == 0) v[0] = 1ull;          // T[empty set] = 1
            }
            // rows hi \ i
            unsigned mm = hi & any;
            while (mm) {
                const int i = __ffs(mm) - 1;
                mm &= mm - 1;
                const unsigned nb = hi ^ (1u << i);
                unsigned long long w[kRow];
#pragma unroll
                for (int z = 0; z < kPairs; z++) {
                    const ulonglong2 x = E[zo_pair<RB>(nb, z)];
                    w[2 * z] = x.x;
                    w[2 * z + 1] = x.y;
                }
#pragma unroll
                for (int lo = 0; lo < kRow; lo++)
                    if ((R[popc_const(lo)] >> (RB + i)) & 1u) v[lo] += w[lo];
            }
            // terms inside the row, in increasing lo
#pragma unroll
            for (int lo = 1; lo < kRow; lo++)
#pragma unroll
                for (int b = 0; b < RB; b++)
                    if (((lo >> b) & 1) && ((R[popc_const(lo)] >> b) & 1u)) v[lo] += v[lo ^ (1 << b)];
#pragma unroll
            for (int z = 0; z < kPairs; z++) {
                const ulonglong2 x = make_ulonglong2(v[2 * z], v[2 * z + 1]);
                E[zo_pair<RB>(hi, z)] = x;
                if (gdst) reinterpret_cast<ulonglong2*>(gdst)[(size_t)hi * kPairs + z] = x;
            }
            if (last && hi == full) {
                unsigned long long* dst = out + (size_t)mc.out_words * out_index;
                dst[0] = v[kRow - 1];
                dst[1] = 0ull;
                if (mc.out_words == 4) { dst[2] = 0ull; dst[3] = 0ull; }
            }
        }
        off += cnt;
        __syncthreads();
    }
}

// Batched 0/1 kernel for orders <= 20 with the register-row chains (chains
// narrower than RB + 1 columns take chain_int).  Same arguments and results as
// sz_batched_int<true, true, THREADS>; the chain tables in the workspace are
// in natural mask order instead of the mask-list order.
template <int THREADS, int RB>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 5 : 2)
sz_batched_zo64(const long long* __restrict__ mats, const ItemDesc* __restrict__ items, int count,
                int m_param, unsigned long long* out, int out_words, int* item_status,
                unsigned long long* workspace, size_t ws_words_per_cta, unsigned* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ int s_width;
    __shared__ int s_pslot[kBinomDim];
    __shared__ unsigned s_obits[kMaxN + 2];
    fill_binom(reinterpret_cast<unsigned*>(smem));
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= count) break;
        const ItemDesc d = items[it];
        const int n = d.n;
        if (threadIdx.x == 0) s_width = decide_width(mats + d.offset, n, true);
        const SmemLayout L = smem_layout(kU64, n, sz_low_for(n, m_param));
        MatCtx mc;
        init_ctx(mc, n, m_param, smem, L);
        mc.out_words = out_words;
        unsigned long long* coef = reinterpret_cast<unsigned long long*>(smem + L.coef_off);
        load_coef_int(mats + d.offset, n, mc.m, coef, reinterpret_cast<unsigned*>(smem + L.rowmask_off));
        __syncthreads();
        const int w = s_width;
        unsigned long long* ws = workspace + (size_t)blockIdx.x * ws_words_per_cta;
        if (mc.m < RB + 1) {
            run_matrix_cta<kU64, true>(mc, smem + L.chain_off, ws, smem + L.coef_off, out, d.out_index,
                                       reinterpret_cast<int*>(smem + L.hinfo_off));
        } else {
            const size_t CW = chain_words(kU64, mc.m);
            const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * CW;
            ulonglong2* E = reinterpret_cast<ulonglong2*>(smem + L.chain_off);
            for (int s = 0; s <= mc.t; s++) {
                const unsigned nslots = (unsigned)binom_calc(mc.t, s);
                unsigned long long* dst_region = ws + (size_t)(s & 1) * layer_words;
                const unsigned long long* src_region = ws + (size_t)((s + 1) & 1) * layer_words;
                const bool last = (s == mc.t);
                for (unsigned slot = 0; slot < nslots; slot++) {
                    zo_chain_setup(mc, coef, unrank_high(slot, s, mc.t, mc.bn), s, s_pslot, s_obits);
                    __syncthreads();
                    chain_zo64<RB>(mc, s, E, src_region, last ? nullptr : dst_region + (size_t)slot * CW,
                                   s_pslot, s_obits, last, out, d.out_index);
                    // every chain ends with __syncthreads()
                }
            }
        }
        if (item_status && threadIdx.x == 0) item_status[d.out_index] = width_status(w);
    }
}

// ---------------------------------------------------------------------------
// One-matrix-at-a-time path, several matrices of one order per launch: one
// launch per layer s, the CTAs stride over the (matrix, chain slot) pairs of
// that layer.  Matrix c of the launch keeps its two layer regions at
// workspace + c * ws_words_per_item.  items == nullptr: one matrix, `single`.
// Each chain is computed exactly as in the batched kernels, so results do not
// depend on how many matrices share a launch.
// ---------------------------------------------------------------------------
template <int THREADS, bool COMPACT>
__global__ void __launch_bounds__(THREADS, THREADS <= 384 ? 2 : 1)
sz_layer_c128(const double2* __restrict__ mats, const ItemDesc* __restrict__ items, ItemDesc single,
              int count, int n, int m_param, int s, double2* out, int* item_status,
              unsigned long long* workspace, size_t ws_words_per_item) {
    extern __shared__ __align__(16) unsigned char smem[];
    fill_binom(reinterpret_cast<unsigned*>(smem));
    const SmemLayout L = smem_layout(kC128, n, sz_low_for(n, m_param));
    MatCtx mc;
    init_ctx(mc, n, m_param, smem, L);
    const size_t CW = chain_words(kC128, mc.m, COMPACT);
    const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * CW;
    const unsigned nslots = (unsigned)binom_calc(mc.t, s);
    const bool last = (s == mc.t);
    const long long tasks = (long long)count * nslots;
    int cur = -1;
    for (long long task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int c = (int)(task / nslots);
        const unsigned slot = (unsigned)(task % nslots);
        const ItemDesc d = items ? items[c] : single;
        if (c != cur) {                 // the same for the whole CTA
            __syncthreads();
            load_coef_c128(mats + d.offset, n, smem + L.coef_off);
            cur = c;
        }
        unsigned long long* ws = workspace + (size_t)c * ws_words_per_item;
        unsigned long long* dst_region = ws + (size_t)(s & 1) * layer_words;
        const unsigned long long* src_region = ws + (size_t)((s + 1) & 1) * layer_words;
        chain_setup(mc, unrank_high(slot, s, mc.t, mc.bn), reinterpret_cast<int*>(smem + L.hinfo_off));
        __syncthreads();
        run_chain<kC128, false, COMPACT>(mc, s, smem + L.chain_off, src_region,
                                         last ? nullptr : dst_region + (size_t)slot * CW, smem + L.coef_off,
                                         last, out, d.out_index);
        if (last && threadIdx.x == 0 && item_status) item_status[d.out_index] = PERM_OK;
    }
}

// ---------------------------------------------------------------------------
// Dataflow form of the layer path (complex, orders up to kLayerSmallN): one
// persistent launch runs every layer of `count` matrices of order n.  Work
// items are (layer s, matrix c, chain slot), numbered in that order and taken
// from an atomic counter.  An item starts once the s predecessor chains it
// reads are done (a flag per chain) and every chain of layer s - 2 is done (a
// counter per layer): three layer regions rotate, and region s mod 3 held layer
// s - 3, which only layer s - 2 reads.  So the first chains of a layer overlap
// the last chains of the one before instead of waiting for a whole launch.
// Every item's dependencies have smaller numbers, so they were taken before by
// CTAs that are running: every wait ends.  Each wait is still bounded (about a
// second of clock), after which the chain is skipped, still marked done, and
// its matrix reports PERM_ETIMEDOUT.
//
// Per matrix the workspace holds the three regions, then one done flag per chain
// of every layer (layer s's at offset sum_{s' < s} C(t, s')), the done counters of
// layers 0..t, and an error flag; all of them zero at launch.
// ---------------------------------------------------------------------------
constexpr int kThreadsFlow = 384;
constexpr long long kFlowWaitCycles = 2000000000ll;   // about one second at the GB300's clock

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin until *p >= need, at most until `start + kFlowWaitCycles`; false on time-out.
__device__ inline bool flow_wait(const int* p, int need, long long start) {
    while (ld_acquire_gpu(p) < need) {
        if (clock64() - start > kFlowWaitCycles) return false;
        __nanosleep(128);
    }
    return true;
}

__host__ __device__ inline size_t flow_layer_words(int n, int m) {
    const int t = n - m;
    return (size_t)binom_calc(t, t / 2) * chain_words(kC128, m);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS <= 256 ? 3 : 2)
sz_flow_c128(const double2* __restrict__ mats, const ItemDesc* __restrict__ items, int count, int n,
             int m_param, double2* out, int* item_status, unsigned long long* workspace,
             size_t ws_words_per_item, unsigned* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_item;
    __shared__ int s_ok;
    fill_binom(reinterpret_cast<unsigned*>(smem));
    const SmemLayout L = smem_layout(kC128, n, sz_low_for(n, m_param));
    MatCtx mc;
    init_ctx(mc, n, m_param, smem, L);
    const int t = mc.t;
    const size_t CW = chain_words(kC128, mc.m);
    const size_t layer_words = flow_layer_words(n, mc.m);
    const unsigned chains = 1u << t;                   // chains of one matrix, all layers
    const unsigned total = (unsigned)count * chains;
    int* hinfo = reinterpret_cast<int*>(smem + L.hinfo_off);
    int cur = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const unsigned i = s_item;
        if (i >= total) break;
        // (layer, matrix, slot) of item i; fb = the layer's first flag in a matrix
        int s = 0;
        unsigned base = 0, fb = 0;
        while (base + (unsigned)count * mc.bn[t * (kBinomDim + 1) + s] <= i) {
            const unsigned cs = mc.bn[t * (kBinomDim + 1) + s];
            base += (unsigned)count * cs;
            fb += cs;
            s++;
        }
        const unsigned nslots = mc.bn[t * (kBinomDim + 1) + s];
        const int c = (int)((i - base) / nslots);
        const unsigned slot = (i - base) % nslots;
        const ItemDesc d = items[c];
        unsigned long long* ws = workspace + (size_t)c * ws_words_per_item;
        int* flags = reinterpret_cast<int*>(ws + 3 * layer_words);
        int* done = flags + chains;                        // layers 0..t
        int* err = done + t + 1;
        chain_setup(mc, unrank_high(slot, s, t, mc.bn), hinfo);
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long start = clock64();
            bool ok = true;
            const unsigned pfb = fb - (s >= 1 ? mc.bn[t * (kBinomDim + 1) + s - 1] : 0u);
            for (int q = 0; q < s && ok; q++) ok = flow_wait(flags + pfb + hinfo[q], 1, start);
            if (ok && s >= 2) ok = flow_wait(done + s - 2, (int)mc.bn[t * (kBinomDim + 1) + s - 2], start);
            if (!ok) atomicExch(err, 1);
            s_ok = ok;
        }
        if (c != cur) {                                    // the same for the whole CTA
            load_coef_c128(mats + d.offset, n, smem + L.coef_off);
            cur = c;
        }
        __syncthreads();
        const bool last = (s == t);
        unsigned long long* dst = ws + (size_t)(s % 3) * layer_words + (size_t)slot * CW;
        const unsigned long long* src = ws + (size_t)((s + 2) % 3) * layer_words;
        if (s_ok) {
            run_chain<kC128, false, false, true>(mc, s, smem + L.chain_off, src, last ? nullptr : dst,
                                                 smem + L.coef_off, last, out, d.out_index);
        }
        // the chain's entries visible to every SM, then its flag and its layer's count
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(done + s, 1);
            st_release_gpu(flags + fb + slot, 1);
            if (last && item_status)
                item_status[d.out_index] = ld_acquire_gpu(err) ? PERM_ETIMEDOUT : PERM_OK;
        }
    }
}

template <bool ZO>
__global__ void __launch_bounds__(kThreadsInt, 3)
sz_layer_int(const long long* __restrict__ mats, const ItemDesc* __restrict__ items, ItemDesc single,
             int count, int n, int m_param, int s, unsigned long long* out, int out_words,
             int* item_status, unsigned long long* workspace, size_t ws_words_per_item) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_width;
    fill_binom(reinterpret_cast<unsigned*>(smem));
    const SmemLayout L = smem_layout(kU128, n, sz_low_for(n, m_param));
    MatCtx mc;
    init_ctx(mc, n, m_param, smem, L);
    mc.out_words = out_words;
    // the workspace is sized for 128-bit chains; 64-bit chains use the same region size
    const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * chain_words(kU128, mc.m);
    const unsigned nslots = (unsigned)binom_calc(mc.t, s);
    const bool last = (s == mc.t);
    const long long tasks = (long long)count * nslots;
    int cur = -1;
    for (long long task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int c = (int)(task / nslots);
        const unsigned slot = (unsigned)(task % nslots);
        const ItemDesc d = items ? items[c] : single;
        if (c != cur) {                 // the same for the whole CTA
            __syncthreads();
            const long long* a = mats + d.offset;
            if (threadIdx.x == 0) s_width = decide_width(a, n, ZO);
            load_coef_int(a, n, mc.m, reinterpret_cast<unsigned long long*>(smem + L.coef_off),
                          reinterpret_cast<unsigned*>(smem + L.rowmask_off));
            cur = c;
        }
        __syncthreads();
        const int w = s_width;
        const int kind = (w == kWidth64) ? kU64 : kU128;
        const size_t CW = chain_words(kind, mc.m);
        unsigned long long* ws = workspace + (size_t)c * ws_words_per_item;
        unsigned long long* dst_region = ws + (size_t)(s & 1) * layer_words;
        const unsigned long long* src_region = ws + (size_t)((s + 1) & 1) * layer_words;
        chain_setup(mc, unrank_high(slot, s, mc.t, mc.bn), reinterpret_cast<int*>(smem + L.hinfo_off));
        __syncthreads();
        unsigned long long* dst = last ? nullptr : dst_region + (size_t)slot * CW;
        if (kind == kU64)
            run_chain<kU64, ZO>(mc, s, smem + L.chain_off, src_region, dst, smem + L.coef_off, last, out,
                                d.out_index);
        else
            run_chain<kU128, ZO>(mc, s, smem + L.chain_off, src_region, dst, smem + L.coef_off, last, out,
                                 d.out_index);
        if (last && threadIdx.x == 0 && item_status) item_status[d.out_index] = width_status(w);
    }
}

__global__ void trivial_kernel(int dtype, const ItemDesc* items, int count, void* out, int out_words,
                               int* item_status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int o = items[i].out_index;
    if (dtype == PERM_C128) {
        reinterpret_cast<double2*>(out)[o] = make_double2(1.0, 0.0);
    } else {
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(out) + (size_t)out_words * o;
        for (int w = 0; w < out_words; w++) dst[w] = w == 0 ? 1ull : 0ull;
    }
    if (item_status) item_status[o] = PERM_OK;
}

// Kernel selection for the batched integer path.
typedef void (*int_batched_fn)(const long long*, const ItemDesc*, int, int, unsigned long long*, int,
                               int*, unsigned long long*, size_t, unsigned*);

// 0/1 batches of order <= 20 take the register-row chains (rows of 2^2
// entries); the LIBPERM_SZ_ZO_ROW=0 experiment knob keeps them on the
// mask-list chains of sz_batched_int.  Same results either way.
bool zo_register_rows() {
    static const bool on = [] {
        const char* v = getenv("LIBPERM_SZ_ZO_ROW");
        return !(v && atoi(v) == 0);
    }();
    return on;
}

template <int T>
int_batched_fn pick_int_batched_t(int dtype, int n_max) {
    const bool zo = dtype == PERM_U01;
    if (zo && n_max <= 20)                                            // 20! < 2^64
        return zo_register_rows() ? sz_batched_zo64<T, 2> : sz_batched_int<true, true, T>;
    if (zo) return sz_batched_int<true, false, T>;
    return sz_batched_int<false, false, T>;
}

int_batched_fn pick_int_batched(int dtype, int n_max, int threads) {
    return threads == 512 ? pick_int_batched_t<512>(dtype, n_max) : pick_int_batched_t<256>(dtype, n_max);
}

int batched_kind(int dtype, int n_max) {
    if (dtype == PERM_C128) return kC128;
    return (dtype == PERM_U01 && n_max <= 20) ? kU64 : kU128;
}

// Allow `fn` the largest dynamic shared memory the device offers, once per
// (device, kernel), so that launches on the hot path make no attribute call.
cudaError_t set_smem(const void* fn, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<int, const void*>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    for (auto& d : done)
        if (d.first == dev && d.second == fn) return cudaSuccess;
    int optin = 0;
    cudaFuncAttributes fa;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (bytes > dyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess) done.emplace_back(dev, fn);
    return e;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

// The mask lists of every chain width m = 1..kMaxLow, ordered by (popcount,
// value), as g_masks holds them.  Filled once into a static host array, so
// uploading it allocates nothing.
unsigned short g_masks_host[kMaskTableLen];
std::once_flag g_masks_host_once;

const unsigned short* mask_table_host() {
    std::call_once(g_masks_host_once, [] {
        int k = 0;
        for (int m = 1; m <= kMaxLow; m++)
            for (int l = 0; l <= m; l++)
                for (unsigned x = 0; x < (1u << m); x++)
                    if (__builtin_popcount(x) == l) g_masks_host[k++] = (unsigned short)x;
    });
    return g_masks_host;
}

}  // namespace

cudaError_t sz_init_tables() {
    // once per device, with that device current
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return cudaSuccess;
    e = cudaMemcpyToSymbol(g_masks, mask_table_host(), sizeof(g_masks_host));
    if (e == cudaSuccess) done.push_back(dev);
    return e;
}

size_t sz_matrix_workspace_bytes(int dtype, int n, int m_param) {
    const int m = sz_low_for(n, m_param);
    const int t = n - m;
    if (t <= 0) return 0;
    // integer chains are sized for 128-bit entries
    const size_t cw = dtype == PERM_C128 ? chain_words(kC128, m, n >= kCompactN) : chain_words(kU128, m);
    return 2 * (size_t)binom_calc(t, t / 2) * cw * 8;
}

int sz_smem_bytes(int dtype, int n, int m_param) {
    const int m = sz_low_for(n, m_param);
    if (dtype == PERM_C128) return smem_layout(kC128, n, m).total;
    return smem_layout(kU128, n, m).total;
}


// Batched complex kernel variants by CTA size.
static const void* c128_batched_fn(int threads) {
    switch (threads) {
        case 256: return (const void*)sz_batched_c128<256>;
        case 512: return (const void*)sz_batched_c128<512>;
        case 768: return (const void*)sz_batched_c128<768>;
        default: return (const void*)sz_batched_c128<384>;
    }
}
int sz_c128_threads_valid(int threads) {
    return threads == 256 || threads == 384 || threads == 512 || threads == 768;
}
int sz_int_threads_valid(int threads) { return threads == 256 || threads == 512; }

// Resident CTAs per SM of the batched kernel for a batch whose largest order is n_max.
int sz_batched_occupancy(int dtype, int n_max, int m_param, int threads) {
    const int m = sz_low_for(n_max, m_param);
    const int kind = batched_kind(dtype, n_max);
    const int smem = smem_layout(kind, n_max, m).total;
    const int ithreads = sz_int_threads_valid(threads) ? threads : kThreadsInt;
    const void* fn = dtype == PERM_C128 ? c128_batched_fn(threads)
                                        : (const void*)pick_int_batched(dtype, n_max, ithreads);
    const int nthr = dtype == PERM_C128 ? threads : ithreads;
    if (set_smem(fn, smem) != cudaSuccess) return 1;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nthr, smem) != cudaSuccess)
        return 1;
    return std::max(1, occ);
}

cudaError_t sz_launch_batched(int dtype, const void* mats, const ItemDesc* items, int count,
                              int n_max, int m, int threads, void* out, int out_words,
                              int* item_status, void* workspace, size_t ws_per_cta, int grid,
                              unsigned* counter, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int mm = sz_low_for(n_max, m);
    const int kind = batched_kind(dtype, n_max);
    const int smem = smem_layout(kind, n_max, mm).total;
    cudaError_t e;
    if (dtype == PERM_C128) {
        const void* fn = c128_batched_fn(threads);
        e = set_smem(fn, smem);
        if (e != cudaSuccess) return e;
        const double2* a0 = (const double2*)mats;
        double2* o0 = (double2*)out;
        unsigned long long* w0 = (unsigned long long*)workspace;
        const size_t wpc = ws_per_cta / 8;
        if (threads == 256)
            sz_batched_c128<256><<<grid, 256, smem, st>>>(a0, items, count, m, o0, item_status, w0, wpc, counter);
        else if (threads == 512)
            sz_batched_c128<512><<<grid, 512, smem, st>>>(a0, items, count, m, o0, item_status, w0, wpc, counter);
        else if (threads == 768)
            sz_batched_c128<768><<<grid, 768, smem, st>>>(a0, items, count, m, o0, item_status, w0, wpc, counter);
        else
            sz_batched_c128<384><<<grid, 384, smem, st>>>(a0, items, count, m, o0, item_status, w0, wpc, counter);
    } else {
        const int ithreads = sz_int_threads_valid(threads) ? threads : kThreadsInt;
        int_batched_fn fn = pick_int_batched(dtype, n_max, ithreads);
        e = set_smem((const void*)fn, smem);
        if (e != cudaSuccess) return e;
        fn<<<grid, ithreads, smem, st>>>((const long long*)mats, items, count, m,
                                            (unsigned long long*)out, out_words, item_status,
                                            (unsigned long long*)workspace, ws_per_cta / 8, counter);
    }
    return cudaGetLastError();
}

namespace {

typedef void (*c128_layer_fn)(const double2*, const ItemDesc*, ItemDesc, int, int, int, int, double2*, int*,
                              unsigned long long*, size_t);

// The complex layer kernel for a CTA size (384, 512 or 768; others: 512) and table kind.
c128_layer_fn pick_c128_layer(int threads, bool compact) {
    if (threads == 384) return compact ? sz_layer_c128<384, true> : sz_layer_c128<384, false>;
    if (threads == 768) return compact ? sz_layer_c128<768, true> : sz_layer_c128<768, false>;
    return compact ? sz_layer_c128<kThreadsC128Single, true> : sz_layer_c128<kThreadsC128Single, false>;
}

// Layers 0..t of `count` matrices of order n (items on the device, or one
// matrix `single` when items == nullptr).
cudaError_t sz_launch_layers_impl(int dtype, const void* mats, const ItemDesc* items, ItemDesc single,
                                  int count, int n, int m, void* out, int out_words, int* item_status,
                                  void* workspace, size_t ws_bytes_per_item, int grid_cap, int threads,
                                  cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int mm = sz_low_for(n, m);
    const int t = n - mm;
    const int smem = sz_smem_bytes(dtype, n, m);
    const c128_layer_fn cfn = pick_c128_layer(threads, n >= kCompactN);
    const void* fn = dtype == PERM_C128 ? (const void*)cfn
                   : (dtype == PERM_U01 ? (const void*)sz_layer_int<true> : (const void*)sz_layer_int<false>);
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    const size_t wpi = ws_bytes_per_item / 8;
    const int cthreads = threads == 384 || threads == 768 ? threads : kThreadsC128Single;
    for (int s = 0; s <= t; s++) {
        const unsigned long long tasks = binom_calc(t, s) * (unsigned long long)count;
        const int grid = (int)std::min<unsigned long long>(tasks, (unsigned long long)grid_cap);
        if (dtype == PERM_C128) {
            cfn<<<grid, cthreads, smem, st>>>((const double2*)mats, items, single, count, n, m, s, (double2*)out,
                                              item_status, (unsigned long long*)workspace, wpi);
        } else if (dtype == PERM_U01) {
            sz_layer_int<true><<<grid, kThreadsInt, smem, st>>>(
                (const long long*)mats, items, single, count, n, m, s, (unsigned long long*)out, out_words,
                item_status, (unsigned long long*)workspace, wpi);
        } else {
            sz_layer_int<false><<<grid, kThreadsInt, smem, st>>>(
                (const long long*)mats, items, single, count, n, m, s, (unsigned long long*)out, out_words,
                item_status, (unsigned long long*)workspace, wpi);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t sz_flow_workspace_bytes(int n, int m_param) {
    const int m = sz_low_for(n, m_param);
    const int t = n - m;
    const size_t bytes = 3 * flow_layer_words(n, m) * 8 + (((size_t)1 << t) + t + 2) * sizeof(int);
    return (bytes + 255) & ~(size_t)255;
}

cudaError_t sz_launch_flow(const void* mats, const ItemDesc* items, int count, int n, int m, void* out,
                           int* item_status, void* workspace, size_t ws_bytes_per_item, unsigned* counter,
                           int num_sms, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (n > kLayerSmallN || ws_bytes_per_item < sz_flow_workspace_bytes(n, m)) return cudaErrorInvalidValue;
    const int mm = sz_low_for(n, m);
    // chains of up to 2^11 entries: three 256-thread CTAs per SM (more chains in flight, and more
    // entries per thread between barriers; measured on GB300: one n = 20 matrix 0.33 ms against
    // 0.35, four n = 22 matrices 1.54 ms against 1.69); wider chains: two 384-thread CTAs
    const int threads = mm <= 11 ? 256 : kThreadsFlow;
    const int grid = (threads == 256 ? 3 : 2) * num_sms;
    const int t = n - mm;
    const size_t flag_off = 3 * flow_layer_words(n, mm) * 8;
    const size_t flag_bytes = (((size_t)1 << t) + t + 2) * sizeof(int);
    cudaError_t e = cudaMemset2DAsync(static_cast<unsigned char*>(workspace) + flag_off, ws_bytes_per_item, 0,
                                      flag_bytes, (size_t)count, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
    const int smem = sz_smem_bytes(PERM_C128, n, m);
    const void* fn = threads == 256 ? (const void*)sz_flow_c128<256> : (const void*)sz_flow_c128<kThreadsFlow>;
    if (e == cudaSuccess) e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    if (threads == 256)
        sz_flow_c128<256><<<grid, 256, smem, st>>>((const double2*)mats, items, count, n, m, (double2*)out,
                                                   item_status, (unsigned long long*)workspace,
                                                   ws_bytes_per_item / 8, counter);
    else
        sz_flow_c128<kThreadsFlow><<<grid, kThreadsFlow, smem, st>>>(
            (const double2*)mats, items, count, n, m, (double2*)out, item_status,
            (unsigned long long*)workspace, ws_bytes_per_item / 8, counter);
    return cudaGetLastError();
}

cudaError_t sz_launch_layers(int dtype, const void* mats, const ItemDesc* items, int count, int n, int m,
                             void* out, int out_words, int* item_status, void* workspace,
                             size_t ws_bytes_per_item, int grid_cap, cudaStream_t st, int threads) {
    return sz_launch_layers_impl(dtype, mats, items, ItemDesc{0, n, 0}, count, n, m, out, out_words,
                                 item_status, workspace, ws_bytes_per_item, grid_cap, threads, st);
}

cudaError_t sz_launch_single(int dtype, const void* mats, long long offset, int n, int m,
                             int out_index, void* out, int out_words, int* item_status,
                             void* workspace, int grid_cap, cudaStream_t st) {
    return sz_launch_layers_impl(dtype, mats, nullptr, ItemDesc{offset, n, out_index}, 1, n, m, out,
                                 out_words, item_status, workspace, 0, grid_cap, 0, st);
}

cudaError_t sz_preload(int dtype) {
    cudaFuncAttributes fa;
    const void* fns[16];
    int k = 0;
    fns[k++] = (const void*)trivial_kernel;
    if (dtype == PERM_C128) {
        fns[k++] = c128_batched_fn(256);
        fns[k++] = c128_batched_fn(384);
        fns[k++] = c128_batched_fn(512);
        fns[k++] = c128_batched_fn(768);
        for (int threads : {384, 512, 768})
            for (bool compact : {false, true}) fns[k++] = (const void*)pick_c128_layer(threads, compact);
        fns[k++] = (const void*)sz_flow_c128<kThreadsFlow>;
        fns[k++] = (const void*)sz_flow_c128<256>;
    } else {
        for (int n_max : {20, 34})
            for (int threads : {256, 512}) fns[k++] = (const void*)pick_int_batched(dtype, n_max, threads);
        fns[k++] = dtype == PERM_U01 ? (const void*)sz_layer_int<true> : (const void*)sz_layer_int<false>;
    }
    for (int i = 0; i < k; i++) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, fns[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_trivial(int dtype, const ItemDesc* items, int count, void* out, int out_words,
                           int* item_status, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    trivial_kernel<<<(count + 127) / 128, 128, 0, st>>>(dtype, items, count, out, out_words, item_status);
    return cudaGetLastError();
}

}  // namespace perm

// ---------------------------------------------------------------------------
// Allocation-free entry point (perm_sz_noalloc).
//
// Some callers cannot call cudaMalloc: a framework whose memory pool owns every
// byte of device memory, or a loop that must not take the implicit device-wide
// synchronisation an allocation can cause.  For them this entry point runs the
// single-matrix Store-zechin path with its chain tables in a fixed scratch
// array that lives in the library's device image instead of a plan.
// ---------------------------------------------------------------------------
namespace perm {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;     // 64 MiB per device
constexpr int kNoAllocLow = 13;                               // chain width used by this path

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchBytes / 8];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

__global__ void noalloc_write_one(int dtype, void* out, int* item_status) {
    if (dtype == PERM_C128) {
        reinterpret_cast<double2*>(out)[0] = make_double2(1.0, 0.0);
    } else {
        reinterpret_cast<unsigned long long*>(out)[0] = 1ull;
        reinterpret_cast<unsigned long long*>(out)[1] = 0ull;
    }
    if (item_status) item_status[0] = PERM_OK;
}

// Once per device, with that device current: the scratch address, and the
// mask table every chain kernel reads (sz_init_tables, the same upload the
// plans use; it copies from a static host array and allocates nothing).
cudaError_t noalloc_setup(int dev, void** scratch) {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (g_noalloc_ptr[dev]) { *scratch = g_noalloc_ptr[dev]; return cudaSuccess; }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = sz_init_tables();
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
    *scratch = p;
    return cudaSuccess;
}

}  // namespace

// Largest order perm_sz_noalloc accepts for a dtype (its chain tables must fit the scratch).
int sz_noalloc_max_n(int dtype) {
    int best = 0;
    for (int n = 1; n <= kMaxNSZ; n++)
        if (sz_matrix_workspace_bytes(dtype, n, kNoAllocLow) <= kNoAllocScratchBytes) best = n;
    return best;
}

}  // namespace perm

extern "C" perm_status perm_sz_noalloc(const void* mat, int n, perm_dtype dtype, void* out,
                                       int* item_status, void* stream) {
    using namespace perm;
    if (dtype != PERM_C128 && dtype != PERM_U01 && dtype != PERM_I64) return PERM_EINVAL;
    if (n < 0 || n > sz_noalloc_max_n(dtype) || !out || (n > 0 && !mat)) return PERM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return PERM_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERM_ECUDA;
    void* scratch = nullptr;
    if (noalloc_setup(dev, &scratch) != cudaSuccess) return PERM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        noalloc_write_one<<<1, 1, 0, st>>>(dtype, out, item_status);
        return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
    }
    const cudaError_t e = sz_launch_single(dtype, mat, 0, n, kNoAllocLow, 0, out, 2, item_status,
                                           scratch, sms, st);
    return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}
