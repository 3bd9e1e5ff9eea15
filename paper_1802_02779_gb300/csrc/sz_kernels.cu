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
// GPU organisation ("chains").  The columns are split into m low columns
// 0..m-1 and t = n-m high columns m..n-1.  Every set S is a pair (H, L) of a
// high part and a low part.  A chain is the 2^m entries (H, L) of one high
// subset H and all low subsets L; inside a chain entries are ordered by |L|,
// then by the colex rank of L.  The recurrence splits into
//     low terms   j in L:  T[(H, L \ j)]  -- the same chain, earlier |L|
//     high terms  h in H:  T[(H \ h, L)]  -- another chain, same position
// so one CTA computes one chain in shared memory level by level (|L| =
// 0..m), gathering low parents from shared memory and streaming high parents,
// coalesced, from the predecessor chains in global memory.  Chains are
// processed in layers of |H| = 0..t; layer s needs only layer s-1.
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
// chosen by decide_width); 0/1 and zero coefficients skip their term.
//
// Summation order for every entry: low columns ascending, then high columns
// ascending, i.e. all columns ascending.  The order depends only on (n, m),
// never on the batch, the grid or the CTA.
#include "perm_internal.cuh"

#include <algorithm>

namespace perm {

namespace {

constexpr int kBinomDim = 24;            // C(x, y) for x < 24 (t <= 21, m <= 15)
constexpr int kThreadsC128 = 512;
constexpr int kThreadsInt = 512;

__host__ __device__ inline unsigned long long binom_calc(int n, int k) {
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned long long r = 1;
    for (int i = 1; i <= k; i++) r = r * (unsigned long long)(n - k + i) / (unsigned long long)i;
    return r;
}

// Shared-memory layout, 16-byte aligned pieces.
struct SmemLayout {
    int binom_off;      // unsigned[kBinomDim][kBinomDim + 1]
    int hinfo_off;      // int[2 * kBinomDim]: predecessor slot, column
    int coef_off;       // coefficient planes (n x n each)
    int chain_off;      // chain planes (2^m each)
    int total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int coef_planes, int chain_planes, int n, int m) {
    SmemLayout s;
    s.binom_off = 0;
    s.hinfo_off = align16(s.binom_off + kBinomDim * (kBinomDim + 1) * 4);
    s.coef_off = align16(s.hinfo_off + 2 * kBinomDim * 4);
    s.chain_off = align16(s.coef_off + coef_planes * n * n * 8);
    s.total = align16(s.chain_off + chain_planes * (1 << m) * 8);
    return s;
}

// Element kinds ------------------------------------------------------------

struct KindC128 { static constexpr int kPlanes = 3; };   // u, v, w (coefficients x, y, s)
struct KindU64 { static constexpr int kPlanes = 1; };
struct KindU128 { static constexpr int kPlanes = 2; };   // low, high words

struct u128 { unsigned long long lo, hi; };

__device__ __forceinline__ u128 u128_mac(u128 acc, unsigned long long c, unsigned long long plo,
                                         unsigned long long phi) {
    // acc + c * (phi:plo)  mod 2^128
    unsigned long long lo = c * plo;
    unsigned long long hi = __umul64hi(c, plo) + c * phi;
    unsigned long long nlo = acc.lo + lo;
    unsigned long long carry = nlo < lo ? 1ull : 0ull;
    return {nlo, acc.hi + hi + carry};
}

// Colex unranking of an l-subset of {0..m-1}: returns the bit mask and
// sum_p C(s_p, p) (the "shifted" rank used for parent indices).
__device__ __forceinline__ unsigned unrank_low(unsigned r, int l, int m, const unsigned* bn,
                                               unsigned& shifted) {
    unsigned mask = 0, tb = 0;
    int c = m - 1;
    for (int p = l - 1; p >= 0; p--) {
        while (bn[c * (kBinomDim + 1) + p + 1] > r) c--;
        mask |= 1u << c;
        r -= bn[c * (kBinomDim + 1) + p + 1];
        tb += bn[c * (kBinomDim + 1) + p];
        c--;
    }
    shifted = tb;
    return mask;
}

// Context of one matrix inside one CTA.
struct MatCtx {
    int n, m, t;
    unsigned chain_len;          // 2^m
    const unsigned* bn;          // smem binomials
    const int* hinfo;            // smem: [0..s) predecessor slots, [kBinomDim..) columns
};

// ---------------------------------------------------------------------------
// One chain (high subset H with |H| = s, slot = colex rank of H among the
// s-subsets of the t high columns).  Writes the chain to `gdst` (global, may
// be null) and, if it is the last chain, the permanent to the output.
// `gprev` is the previous layer's region (chains of |H| = s-1).
// ---------------------------------------------------------------------------
template <class Kind>
__device__ void process_chain(const MatCtx& mc, unsigned Hmask, int s, unsigned long long* chain_smem,
                              const unsigned long long* gprev, unsigned long long* gdst,
                              const void* coef_smem, bool last, void* out, int out_index);

// Predecessor info for chain H: for the p-th high element h_p (ascending),
// the slot of H \ h_p among the (s-1)-subsets and the matrix column m + h_p.
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
            hinfo[kBinomDim + p] = mc.m + hs[p];
        }
    }
}

// ---- complex128 ------------------------------------------------------------
template <>
__device__ void process_chain<KindC128>(const MatCtx& mc, unsigned Hmask, int s,
                                        unsigned long long* chain_smem_u,
                                        const unsigned long long* gprev_u,
                                        unsigned long long* gdst_u, const void* coef_smem,
                                        bool last, void* out, int out_index) {
    const int n = mc.n, m = mc.m;
    const unsigned CL = mc.chain_len;
    double* ch = reinterpret_cast<double*>(chain_smem_u);
    const double* gprev = reinterpret_cast<const double*>(gprev_u);
    double* gdst = reinterpret_cast<double*>(gdst_u);
    const double* cx = reinterpret_cast<const double*>(coef_smem);
    const double* cy = cx + n * n;
    const double* cs = cy + n * n;
    const unsigned* bn = mc.bn;
    const int* hslot = mc.hinfo;
    const int* hcol = mc.hinfo + kBinomDim;

    unsigned off_prev = 0, off = 0;
    for (int l = 0; l <= m; l++) {
        const unsigned cnt = bn[m * (kBinomDim + 1) + l];
        const int k = s + l;
        const int row = k - 1;
        for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
            const unsigned idx = off + r;
            double u, v, w;
            if (k == 0) {
                u = 1.0; v = 0.0; w = 1.0;
            } else if (k == 1) {
                // the single column of S
                int col;
                if (l == 1) { unsigned tb; col = __ffs(unrank_low(r, 1, m, bn, tb)) - 1; }
                else col = hcol[0];
                u = cx[col]; v = cy[col]; w = cs[col];
            } else if (k == n) {
                // the permanent: double-double, four-product complex form
                dd2 re = {0.0, 0.0}, im = {0.0, 0.0};
                unsigned tb;
                unsigned mask = unrank_low(r, l, m, bn, tb);
                unsigned A = 0, Bp = 0;
                int p = 0;
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const unsigned pidx = off_prev + A + (tb - Bp - bn[j * (kBinomDim + 1) + p]);
                    A += bn[j * (kBinomDim + 1) + p + 1];
                    Bp += bn[j * (kBinomDim + 1) + p];
                    p++;
                    const double x = cx[row * n + j], y = cy[row * n + j];
                    const double pu = ch[pidx], pv = ch[CL + pidx];
                    re = dd_add_prod(re, x, pu);
                    re = dd_add_prod(re, -y, pv);
                    im = dd_add_prod(im, x, pv);
                    im = dd_add_prod(im, y, pu);
                }
                for (int q = 0; q < s; q++) {
                    const double* pc = gprev + (size_t)hslot[q] * 3 * CL;
                    const int col = hcol[q];
                    const double x = cx[row * n + col], y = cy[row * n + col];
                    const double pu = pc[idx], pv = pc[CL + idx];
                    re = dd_add_prod(re, x, pu);
                    re = dd_add_prod(re, -y, pv);
                    im = dd_add_prod(im, x, pv);
                    im = dd_add_prod(im, y, pu);
                }
                u = dd_round(re); v = dd_round(im); w = __dadd_rn(u, v);
            } else {
                double P1 = 0.0, P2 = 0.0, P3 = 0.0;
                unsigned tb;
                unsigned mask = unrank_low(r, l, m, bn, tb);
                unsigned A = 0, Bp = 0;
                int p = 0;
                const double* rx = cx + row * n;
                const double* ry = cy + row * n;
                const double* rs = cs + row * n;
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const unsigned pidx = off_prev + A + (tb - Bp - bn[j * (kBinomDim + 1) + p]);
                    A += bn[j * (kBinomDim + 1) + p + 1];
                    Bp += bn[j * (kBinomDim + 1) + p];
                    p++;
                    P1 = __fma_rn(rx[j], ch[pidx], P1);
                    P2 = __fma_rn(ry[j], ch[CL + pidx], P2);
                    P3 = __fma_rn(rs[j], ch[2 * CL + pidx], P3);
                }
                // high terms: predecessor chains, same position; prefetch in groups of 4
                int q = 0;
                for (; q + 4 <= s; q += 4) {
                    double gu[4], gv[4], gw[4];
#pragma unroll
                    for (int z = 0; z < 4; z++) {
                        const double* pc = gprev + (size_t)hslot[q + z] * 3 * CL + idx;
                        gu[z] = __ldg(pc);
                        gv[z] = __ldg(pc + CL);
                        gw[z] = __ldg(pc + 2 * CL);
                    }
#pragma unroll
                    for (int z = 0; z < 4; z++) {
                        const int col = hcol[q + z];
                        P1 = __fma_rn(rx[col], gu[z], P1);
                        P2 = __fma_rn(ry[col], gv[z], P2);
                        P3 = __fma_rn(rs[col], gw[z], P3);
                    }
                }
                for (; q < s; q++) {
                    const double* pc = gprev + (size_t)hslot[q] * 3 * CL + idx;
                    const int col = hcol[q];
                    P1 = __fma_rn(rx[col], __ldg(pc), P1);
                    P2 = __fma_rn(ry[col], __ldg(pc + CL), P2);
                    P3 = __fma_rn(rs[col], __ldg(pc + 2 * CL), P3);
                }
                u = __dsub_rn(P1, P2);
                v = __dsub_rn(__dsub_rn(P3, P1), P2);
                w = __dadd_rn(u, v);
            }
            ch[idx] = u; ch[CL + idx] = v; ch[2 * CL + idx] = w;
            if (gdst) { gdst[idx] = u; gdst[CL + idx] = v; gdst[2 * CL + idx] = w; }
            if (last && l == m) {
                reinterpret_cast<double2*>(out)[out_index] = make_double2(u, v);
            }
        }
        off_prev = off;
        off += cnt;
        __syncthreads();
    }
}

// ---- integers modulo 2^64 --------------------------------------------------
template <>
__device__ void process_chain<KindU64>(const MatCtx& mc, unsigned Hmask, int s,
                                       unsigned long long* ch, const unsigned long long* gprev,
                                       unsigned long long* gdst, const void* coef_smem, bool last,
                                       void* out, int out_index) {
    const int n = mc.n, m = mc.m;
    const unsigned CL = mc.chain_len;
    const unsigned long long* co = reinterpret_cast<const unsigned long long*>(coef_smem);
    const unsigned* bn = mc.bn;
    const int* hslot = mc.hinfo;
    const int* hcol = mc.hinfo + kBinomDim;
    unsigned off_prev = 0, off = 0;
    for (int l = 0; l <= m; l++) {
        const unsigned cnt = bn[m * (kBinomDim + 1) + l];
        const int k = s + l;
        const unsigned long long* rc = co + (k >= 1 ? (k - 1) * n : 0);
        for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
            const unsigned idx = off + r;
            unsigned long long val;
            if (k == 0) {
                val = 1ull;
            } else if (k == 1) {
                int col;
                if (l == 1) { unsigned tb; col = __ffs(unrank_low(r, 1, m, bn, tb)) - 1; }
                else col = hcol[0];
                val = co[col];
            } else {
                val = 0ull;
                unsigned tb;
                unsigned mask = unrank_low(r, l, m, bn, tb);
                unsigned A = 0, Bp = 0;
                int p = 0;
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const unsigned pidx = off_prev + A + (tb - Bp - bn[j * (kBinomDim + 1) + p]);
                    A += bn[j * (kBinomDim + 1) + p + 1];
                    Bp += bn[j * (kBinomDim + 1) + p];
                    p++;
                    const unsigned long long c = rc[j];
                    if (c) val += c * ch[pidx];
                }
                for (int q = 0; q < s; q++) {
                    const unsigned long long c = rc[hcol[q]];
                    if (c) val += c * __ldg(gprev + (size_t)hslot[q] * CL + idx);
                }
            }
            ch[idx] = val;
            if (gdst) gdst[idx] = val;
            if (last && l == m) {
                unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
                o[2 * out_index] = val;
                o[2 * out_index + 1] = 0ull;
            }
        }
        off_prev = off;
        off += cnt;
        __syncthreads();
    }
}

// ---- integers modulo 2^128 -------------------------------------------------
template <>
__device__ void process_chain<KindU128>(const MatCtx& mc, unsigned Hmask, int s,
                                        unsigned long long* ch, const unsigned long long* gprev,
                                        unsigned long long* gdst, const void* coef_smem, bool last,
                                        void* out, int out_index) {
    const int n = mc.n, m = mc.m;
    const unsigned CL = mc.chain_len;
    const unsigned long long* co = reinterpret_cast<const unsigned long long*>(coef_smem);
    const unsigned* bn = mc.bn;
    const int* hslot = mc.hinfo;
    const int* hcol = mc.hinfo + kBinomDim;
    unsigned off_prev = 0, off = 0;
    for (int l = 0; l <= m; l++) {
        const unsigned cnt = bn[m * (kBinomDim + 1) + l];
        const int k = s + l;
        const unsigned long long* rc = co + (k >= 1 ? (k - 1) * n : 0);
        for (unsigned r = threadIdx.x; r < cnt; r += blockDim.x) {
            const unsigned idx = off + r;
            u128 val;
            if (k == 0) {
                val = {1ull, 0ull};
            } else if (k == 1) {
                int col;
                if (l == 1) { unsigned tb; col = __ffs(unrank_low(r, 1, m, bn, tb)) - 1; }
                else col = hcol[0];
                val = {co[col], 0ull};
            } else {
                val = {0ull, 0ull};
                unsigned tb;
                unsigned mask = unrank_low(r, l, m, bn, tb);
                unsigned A = 0, Bp = 0;
                int p = 0;
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const unsigned pidx = off_prev + A + (tb - Bp - bn[j * (kBinomDim + 1) + p]);
                    A += bn[j * (kBinomDim + 1) + p + 1];
                    Bp += bn[j * (kBinomDim + 1) + p];
                    p++;
                    const unsigned long long c = rc[j];
                    if (c) val = u128_mac(val, c, ch[pidx], ch[CL + pidx]);
                }
                for (int q = 0; q < s; q++) {
                    const unsigned long long c = rc[hcol[q]];
                    if (c) {
                        const unsigned long long* pc = gprev + (size_t)hslot[q] * 2 * CL + idx;
                        val = u128_mac(val, c, __ldg(pc), __ldg(pc + CL));
                    }
                }
            }
            ch[idx] = val.lo; ch[CL + idx] = val.hi;
            if (gdst) { gdst[idx] = val.lo; gdst[CL + idx] = val.hi; }
            if (last && l == m) {
                unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
                o[2 * out_index] = val.lo;
                o[2 * out_index + 1] = val.hi;
            }
        }
        off_prev = off;
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

// Load the coefficient planes of one matrix into shared memory.
__device__ inline void load_coef_c128(const double2* a, int n, double* coef) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const double2 z = a[e];
        coef[e] = z.x;
        coef[n * n + e] = z.y;
        coef[2 * n * n + e] = __dadd_rn(z.x, z.y);
    }
}
__device__ inline void load_coef_int(const long long* a, int n, unsigned long long* coef) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) coef[e] = (unsigned long long)a[e];
}

// All chains of one matrix, inside one CTA (batched mode).
template <class Kind>
__device__ void run_matrix_cta(MatCtx& mc, unsigned long long* chain_smem, unsigned long long* ws,
                               const void* coef, void* out, int out_index, int* hinfo_smem) {
    const size_t CW = (size_t)Kind::kPlanes * mc.chain_len;
    const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * CW;
    for (int s = 0; s <= mc.t; s++) {
        const unsigned nslots = (unsigned)binom_calc(mc.t, s);
        unsigned long long* dst_region = ws + (size_t)(s & 1) * layer_words;
        const unsigned long long* src_region = ws + (size_t)((s + 1) & 1) * layer_words;
        for (unsigned slot = 0; slot < nslots; slot++) {
            const unsigned H = unrank_high(slot, s, mc.t, mc.bn);
            chain_setup(mc, H, hinfo_smem);
            __syncthreads();
            const bool last = (s == mc.t);
            process_chain<Kind>(mc, H, s, chain_smem, src_region,
                                last ? nullptr : dst_region + (size_t)slot * CW, coef, last, out,
                                out_index);
            // process_chain ends with __syncthreads()
        }
    }
}

template <class Kind>
__device__ void write_status(int* item_status, int idx, int st) {
    if (item_status && threadIdx.x == 0) item_status[idx] = st;
}

// ---------------------------------------------------------------------------
// Batched kernels: one CTA per matrix, persistent over the item list.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreadsC128)
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
        MatCtx mc;
        mc.n = n;
        mc.m = sz_low_for(n, m_param);
        mc.t = n - mc.m;
        mc.chain_len = 1u << mc.m;
        const SmemLayout L = smem_layout(3, 3, n, mc.m);
        mc.bn = reinterpret_cast<const unsigned*>(smem + L.binom_off);
        mc.hinfo = reinterpret_cast<const int*>(smem + L.hinfo_off);
        double* coef = reinterpret_cast<double*>(smem + L.coef_off);
        load_coef_c128(mats + d.offset, n, coef);
        __syncthreads();
        run_matrix_cta<KindC128>(mc, reinterpret_cast<unsigned long long*>(smem + L.chain_off),
                                 workspace + (size_t)blockIdx.x * ws_words_per_cta, coef, out,
                                 d.out_index, reinterpret_cast<int*>(smem + L.hinfo_off));
        write_status<KindC128>(item_status, d.out_index, PERM_OK);
    }
}

__global__ void __launch_bounds__(kThreadsInt)
sz_batched_int(const long long* __restrict__ mats, const ItemDesc* __restrict__ items, int count,
               int m_param, int zero_one, unsigned long long* out, int* item_status,
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
        if (threadIdx.x == 0) s_width = decide_width(mats + d.offset, n, zero_one != 0);
        MatCtx mc;
        mc.n = n;
        mc.m = sz_low_for(n, m_param);
        mc.t = n - mc.m;
        mc.chain_len = 1u << mc.m;
        const SmemLayout L = smem_layout(1, 2, n, mc.m);
        mc.bn = reinterpret_cast<const unsigned*>(smem + L.binom_off);
        mc.hinfo = reinterpret_cast<const int*>(smem + L.hinfo_off);
        unsigned long long* coef = reinterpret_cast<unsigned long long*>(smem + L.coef_off);
        load_coef_int(mats + d.offset, n, coef);
        __syncthreads();
        const int w = s_width;
        unsigned long long* ws = workspace + (size_t)blockIdx.x * ws_words_per_cta;
        unsigned long long* chain = reinterpret_cast<unsigned long long*>(smem + L.chain_off);
        int* hinfo = reinterpret_cast<int*>(smem + L.hinfo_off);
        if (w == kWidth64)
            run_matrix_cta<KindU64>(mc, chain, ws, coef, out, d.out_index, hinfo);
        else
            run_matrix_cta<KindU128>(mc, chain, ws, coef, out, d.out_index, hinfo);
        write_status<KindU64>(item_status, d.out_index, width_status(w));
    }
}

// ---------------------------------------------------------------------------
// Single-matrix kernels: one launch per layer s; CTAs stride over the slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreadsC128)
sz_layer_c128(const double2* __restrict__ a, int n, int m, int s, double2* out, int out_index,
              int* item_status, unsigned long long* workspace) {
    extern __shared__ __align__(16) unsigned char smem[];
    fill_binom(reinterpret_cast<unsigned*>(smem));
    MatCtx mc;
    mc.n = n;
    mc.m = m;
    mc.t = n - m;
    mc.chain_len = 1u << m;
    const SmemLayout L = smem_layout(3, 3, n, m);
    mc.bn = reinterpret_cast<const unsigned*>(smem + L.binom_off);
    mc.hinfo = reinterpret_cast<const int*>(smem + L.hinfo_off);
    double* coef = reinterpret_cast<double*>(smem + L.coef_off);
    load_coef_c128(a, n, coef);
    __syncthreads();
    const size_t CW = (size_t)3 * mc.chain_len;
    const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * CW;
    unsigned long long* dst_region = workspace + (size_t)(s & 1) * layer_words;
    const unsigned long long* src_region = workspace + (size_t)((s + 1) & 1) * layer_words;
    const unsigned nslots = (unsigned)binom_calc(mc.t, s);
    const bool last = (s == mc.t);
    for (unsigned slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const unsigned H = unrank_high(slot, s, mc.t, mc.bn);
        chain_setup(mc, H, reinterpret_cast<int*>(smem + L.hinfo_off));
        __syncthreads();
        process_chain<KindC128>(mc, H, s, reinterpret_cast<unsigned long long*>(smem + L.chain_off),
                                src_region, last ? nullptr : dst_region + (size_t)slot * CW, coef,
                                last, out, out_index);
    }
    if (last && blockIdx.x == 0 && threadIdx.x == 0 && item_status) item_status[out_index] = PERM_OK;
}

__global__ void __launch_bounds__(kThreadsInt)
sz_layer_int(const long long* __restrict__ a, int n, int m, int s, int zero_one,
             unsigned long long* out, int out_index, int* item_status,
             unsigned long long* workspace) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_width;
    fill_binom(reinterpret_cast<unsigned*>(smem));
    if (threadIdx.x == 0) s_width = decide_width(a, n, zero_one != 0);
    MatCtx mc;
    mc.n = n;
    mc.m = m;
    mc.t = n - m;
    mc.chain_len = 1u << m;
    const SmemLayout L = smem_layout(1, 2, n, m);
    mc.bn = reinterpret_cast<const unsigned*>(smem + L.binom_off);
    mc.hinfo = reinterpret_cast<const int*>(smem + L.hinfo_off);
    unsigned long long* coef = reinterpret_cast<unsigned long long*>(smem + L.coef_off);
    load_coef_int(a, n, coef);
    __syncthreads();
    const int w = s_width;
    const int planes = (w == kWidth64) ? 1 : 2;
    const size_t CW = (size_t)planes * mc.chain_len;
    // the workspace is sized for two planes; one-plane chains use the same stride
    const size_t layer_words = (size_t)binom_calc(mc.t, mc.t / 2) * 2 * mc.chain_len;
    unsigned long long* dst_region = workspace + (size_t)(s & 1) * layer_words;
    const unsigned long long* src_region = workspace + (size_t)((s + 1) & 1) * layer_words;
    const unsigned nslots = (unsigned)binom_calc(mc.t, s);
    const bool last = (s == mc.t);
    for (unsigned slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const unsigned H = unrank_high(slot, s, mc.t, mc.bn);
        chain_setup(mc, H, reinterpret_cast<int*>(smem + L.hinfo_off));
        __syncthreads();
        unsigned long long* chain = reinterpret_cast<unsigned long long*>(smem + L.chain_off);
        unsigned long long* dst = last ? nullptr : dst_region + (size_t)slot * CW;
        if (w == kWidth64)
            process_chain<KindU64>(mc, H, s, chain, src_region, dst, coef, last, out, out_index);
        else
            process_chain<KindU128>(mc, H, s, chain, src_region, dst, coef, last, out, out_index);
    }
    if (last && blockIdx.x == 0 && threadIdx.x == 0 && item_status)
        item_status[out_index] = width_status(w);
}

__global__ void trivial_kernel(int dtype, const ItemDesc* items, int count, void* out,
                               int* item_status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int o = items[i].out_index;
    if (dtype == PERM_C128) {
        reinterpret_cast<double2*>(out)[o] = make_double2(1.0, 0.0);
    } else {
        reinterpret_cast<unsigned long long*>(out)[2 * o] = 1ull;
        reinterpret_cast<unsigned long long*>(out)[2 * o + 1] = 0ull;
    }
    if (item_status) item_status[o] = PERM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
unsigned long long binom_host(int n, int k) { return binom_calc(n, k); }

size_t sz_chain_words(int dtype, int m) {
    const int planes = dtype == PERM_C128 ? 3 : 2;   // integer chains sized for 128-bit
    return (size_t)planes << m;
}

size_t sz_matrix_workspace_bytes(int dtype, int n, int m_param) {
    const int m = sz_low_for(n, m_param);
    const int t = n - m;
    if (t <= 0) return 0;
    return 2 * (size_t)binom_calc(t, t / 2) * sz_chain_words(dtype, m) * 8;
}

int sz_smem_bytes(int dtype, int n, int m) {
    if (dtype == PERM_C128) return smem_layout(3, 3, n, m).total;
    return smem_layout(1, 2, n, m).total;
}

int sz_threads(int dtype) { return dtype == PERM_C128 ? kThreadsC128 : kThreadsInt; }

static cudaError_t set_smem(const void* fn, int bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t sz_launch_batched(int dtype, const void* mats, const ItemDesc* items, int count,
                              int n_max, int m, void* out, int* item_status, void* workspace,
                              size_t ws_per_cta, int grid, unsigned* counter, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int mm = sz_low_for(n_max, m);
    const int smem = sz_smem_bytes(dtype, n_max, mm);
    cudaError_t e;
    if (dtype == PERM_C128) {
        e = set_smem((const void*)sz_batched_c128, smem);
        if (e != cudaSuccess) return e;
        sz_batched_c128<<<grid, kThreadsC128, smem, st>>>(
            (const double2*)mats, items, count, m, (double2*)out, item_status,
            (unsigned long long*)workspace, ws_per_cta / 8, counter);
    } else {
        e = set_smem((const void*)sz_batched_int, smem);
        if (e != cudaSuccess) return e;
        sz_batched_int<<<grid, kThreadsInt, smem, st>>>(
            (const long long*)mats, items, count, m, dtype == PERM_U01 ? 1 : 0,
            (unsigned long long*)out, item_status, (unsigned long long*)workspace,
            ws_per_cta / 8, counter);
    }
    return cudaGetLastError();
}

cudaError_t sz_launch_single(int dtype, const void* mats, long long offset, int n, int m,
                             int out_index, void* out, int* item_status, void* workspace,
                             int grid_cap, cudaStream_t st) {
    const int mm = sz_low_for(n, m);
    const int t = n - mm;
    const int smem = sz_smem_bytes(dtype, n, mm);
    cudaError_t e;
    if (dtype == PERM_C128) e = set_smem((const void*)sz_layer_c128, smem);
    else e = set_smem((const void*)sz_layer_int, smem);
    if (e != cudaSuccess) return e;
    for (int s = 0; s <= t; s++) {
        const int grid = (int)std::min<unsigned long long>(binom_calc(t, s), (unsigned long long)grid_cap);
        if (dtype == PERM_C128) {
            sz_layer_c128<<<grid, kThreadsC128, smem, st>>>(
                (const double2*)mats + offset, n, mm, s, (double2*)out, out_index, item_status,
                (unsigned long long*)workspace);
        } else {
            sz_layer_int<<<grid, kThreadsInt, smem, st>>>(
                (const long long*)mats + offset, n, mm, s, dtype == PERM_U01 ? 1 : 0,
                (unsigned long long*)out, out_index, item_status, (unsigned long long*)workspace);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_trivial(int dtype, const ItemDesc* items, int count, void* out,
                           int* item_status, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    trivial_kernel<<<(count + 127) / 128, 128, 0, st>>>(dtype, items, count, out, item_status);
    return cudaGetLastError();
}

}  // namespace perm
